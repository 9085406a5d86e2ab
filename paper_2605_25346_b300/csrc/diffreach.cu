// Host side of the C ABI declared in include/diffreach.h: context, uploads, launch logic.
#include <cuda_runtime.h>

#include <algorithm>
#include <limits>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/diffreach.h"
#include "common.cuh"
#include "fused_core.cuh"
#include "fused_bwd.cuh"
#include "fused_multi.cuh"
#include "fused_warp.cuh"
#include "tc_gemm.cuh"
#include "tc_gemm_persistent.cuh"
#include "wide.cuh"
#include "wide_bwd.cuh"


struct dr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t launches = 0;
    size_t owned = 0;

    bool has_ctrl = false;
    NetDesc net{};
    float* dW = nullptr;
    float* db = nullptr;

    bool has_dyn = false;
    double* dA = nullptr;
    double* dB = nullptr;
    double* de = nullptr;

    int64_t D = 0;
    double* dlo0 = nullptr;
    double* dhi0 = nullptr;

    int64_t nnz = 0;
    int64_t* dsp_row = nullptr;
    SplitRec* dsp = nullptr;
    float* dbeta = nullptr;

    int H = 0;
    dr_options opt{};

    float* dalpha = nullptr;  // [D][H][hidden]
    bool alpha_set = false;

    double* deoff = nullptr;    // [D][H][n] per-step offsets of the dynamics (null: none)
    double* dgshift = nullptr;  // [D][H+1][n] shift gradient written by the last dr_backward
    bool gshift_valid = false;
    float* dgth = nullptr;       // per-domain slices of dV/dtheta of one backward chunk
    size_t gth_bytes = 0;
    double* dgth_part = nullptr; // [kThetaGroups][nparams] partial sums over the slices
    double* dgtheta = nullptr;   // [nparams] dV/dtheta (W packed, then b) of the last dr_backward
    bool gtheta_valid = false;

    // library-owned outputs / scratch
    double* dout_lo = nullptr;
    double* dout_hi = nullptr;
    double* dV = nullptr;
    uint32_t* dstatus = nullptr;
    double* dhull = nullptr;
    double* dtape = nullptr;
    size_t tape_bytes = 0;
    size_t out_bytes = 0;
    // refinement / adjoint scratch
    float* dgalpha = nullptr;
    float* dgbeta = nullptr;
    float* dbest_alpha = nullptr;
    float* dbest_beta = nullptr;
    double* dbestV = nullptr;
    double* dVhist = nullptr;
    int* dhist_slot = nullptr;  // next V history entry of dr_optimize_slopes (device-side counter)
    double* dwlo = nullptr;
    double* dwhi = nullptr;
    // transposed TF32 parts of every layer for the tensor-core chain: layer l -> [n_{l-1}][ru32(n_l)]
    float* dWTh = nullptr;
    float* dWTl = nullptr;
    int64_t WToff[DR_MAXL] = {};
    // W_2 and [W_2^+; W_2^-] as blocked TF32 parts (left operands of the target-2 GEMMs), rows
    // padded to 128, K = ru32(n_1); null for a one-layer controller
    float *dA2h = nullptr, *dA2l = nullptr, *dA2ph = nullptr, *dA2pl = nullptr;
    // for the staged reverse sweep: every layer W_l as TF32 parts [n_l][ru32(n_{l-1})] (right operand
    // of the reverse chain GEMMs) and in the kept-level layout (blocked as the operands, rows padded to
    // 128: the shared top level of the reverse chain)
    float *dWRh = nullptr, *dWRl = nullptr, *dWlev = nullptr;
    int64_t WRoff[DR_MAXL] = {}, WLoff[DR_MAXL] = {};
    // staged reverse sweep: keep store and adjoint scratch of one chunk, split values h
    void* kscratch = nullptr;
    size_t kscratch_bytes = 0;
    float* dsph = nullptr;
    int64_t sph_n = 0;
    int* derr = nullptr;
    // per-CTA global slabs for the fused kernels on wide controllers (tape runs), and the one padded
    // weight copy they share
    unsigned char* gslab = nullptr;
    size_t gslab_bytes = 0;
    float* dWpad = nullptr;
    // staged (wide) path chunk scratch
    void* wscratch = nullptr;
    size_t wscratch_bytes = 0;
    int wDc = 0;
    int wLanes = 0;
    // CUDA-graph replay of dr_compute_bounds: any device allocation or free bumps `epoch`; a graph is
    // captured on the second call with the same (epoch, slope mode, hull) and replayed while they hold
    uint64_t epoch = 1;
    cudaGraphExec_t gexec = nullptr;
    uint64_t g_epoch = 0, seen_epoch = 0;
    int g_mode = -1, g_hull = -1, seen_mode = -1, seen_hull = -1;
    int64_t graph_launches = 0, graph_replays = 0;
    bool capturing = false, graphs_broken = false, g_check_tc = false, last_tc = false;
    // extra streams (and fork/join events) for the staged path's independent domain lanes
    static constexpr int kMaxLanes = 4;
    cudaStream_t aux[kMaxLanes] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kMaxLanes] = {};
    // per-launch timing of the tensor-core GEMMs (dr_options.timing): event pairs not yet read, a
    // pool of reusable events and the per-class totals
    struct KtPending {
        int cls;
        int64_t rows;
        cudaEvent_t e0, e1;
        double flop;
    };
    struct KtDone {
        int cls;
        int64_t rows;
        double ms, flop;
    };
    std::vector<KtPending> kt_pending;
    std::vector<KtDone> kt_done;
    std::vector<cudaEvent_t> kt_pool;
};

static thread_local std::string g_create_err;

static int fail(dr_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_err = buf;
    return code;
}

#define CUDA_TRY(ctx, call)                                                                       \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(ctx, DR_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static void dev_free(dr_ctx* c, void*& p, size_t bytes) {
    if (p) {
        c->epoch++;
        cudaFree(p);
        c->owned -= std::min(c->owned, bytes);
        p = nullptr;
    }
}

template <typename T>
static int dev_alloc(dr_ctx* c, T*& p, size_t count) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    if (c->opt.mem_cap_bytes > 0 && c->owned + bytes > (size_t)c->opt.mem_cap_bytes)
        return fail(c, DR_ERR_OOM, "allocation of %zu bytes exceeds the memory cap (%lld bytes, %zu owned)", bytes,
                    (long long)c->opt.mem_cap_bytes, c->owned);
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, DR_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->epoch++;
    c->owned += bytes;
    p = reinterpret_cast<T*>(q);
    return DR_OK;
}

#define TRY(x)                 \
    do {                       \
        int r_ = (x);          \
        if (r_ != DR_OK) return r_; \
    } while (0)

static dr_options default_options() {
    dr_options o;
    memset(&o, 0, sizeof(o));
    o.slope_mode = DR_SLOPE_CHORD;
    o.precision = DR_PREC_AUTO;
    o.margin_rho = 0.0;
    o.box_margin = std::ldexp(1.0, -18);
    o.chunk_domains = 0;
    o.mem_cap_bytes = 0;
    return o;
}

// ------------------------------------------------------------------------------------------------
// fused-path layout
// ------------------------------------------------------------------------------------------------

static const int kMaxSmem = 227 * 1024;

// top_adjoint: the Lambda-adjoint buffers also hold each target's top chain level (n_l x n_{l-1}),
// which the weight gradient reads and the slab kernels' tiled products use as scratch; a backward
// layout that does not fit shared memory (slab mode) always includes it.
static FusedLayout fused_layout(const NetDesc& N, bool backward = false, bool top_adjoint = false) {
    FusedLayout Y;
    memset(&Y, 0, sizeof(Y));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 15) & ~size_t(15);
        const size_t r = off;
        off += bytes;
        return (int)r;
    };
    const int n = N.n, m = N.m;
    for (int l = 0; l < N.L; ++l) Y.Ws[l] = take(sizeof(float) * N.w[l + 1] * odd_ld(N.w[l]));
    int nb = 0;
    for (int l = 0; l < N.L; ++l) nb += N.w[l + 1];
    Y.bs = take(sizeof(float) * nb);
    Y.A = take(sizeof(double) * n * n);
    Y.B = take(sizeof(double) * n * m);
    Y.e = take(sizeof(double) * n);
    Y.c = take(sizeof(double) * n);
    Y.P = take(sizeof(double) * n * n);
    Y.Ilo = take(sizeof(double) * n);
    Y.Ihi = take(sizeof(double) * n);
    Y.v = take(sizeof(double) * n);
    Y.w = take(sizeof(double) * 2);
    Y.cn = take(sizeof(double) * n);
    Y.Pn = take(sizeof(double) * std::max(n * n, 64));
    Y.Ilon = take(sizeof(double) * n);
    Y.Ihin = take(sizeof(double) * n);
    Y.cf = take(sizeof(float) * n);
    Y.Pf = take(sizeof(float) * n * n);
    Y.Ilof = take(sizeof(float) * n);
    Y.Ihif = take(sizeof(float) * n);
    Y.vf = take(sizeof(float) * (n + 1));
    const int hid = std::max(N.hidden, 1);
    Y.hl = take(sizeof(float) * hid);
    Y.hu = take(sizeof(float) * hid);
    Y.hs = take(sizeof(float) * hid);
    Y.hd = take(sizeof(float) * hid);
    if (backward) {
        Y.hl0 = take(sizeof(float) * hid);
        Y.hu0 = take(sizeof(float) * hid);
    } else {
        Y.hl0 = Y.hl;
        Y.hu0 = Y.hu;
    }
    Y.klo = take(sizeof(float) * N.maxw);
    Y.khi = take(sizeof(float) * N.maxw);
    // per-domain chain buffers: target l, after level m the matrix is n_l x odd_ld(n_{m-1})
    size_t lam = 1;
    for (int l = 2; l <= N.L; ++l)
        for (int k = 0; k <= l - 2; ++k) lam = std::max(lam, (size_t)N.w[l] * odd_ld(N.w[k]));
    Y.lam0 = take(sizeof(float) * lam);
    Y.lam1 = take(sizeof(float) * lam);
    Y.G = take(sizeof(float) * N.maxw * odd_ld(n));
    Y.a = take(sizeof(float) * N.maxw);
    Y.Rlo = take(sizeof(float) * N.maxw);
    Y.Rhi = take(sizeof(float) * N.maxw);
    Y.S = take(sizeof(float) * N.maxw);
    Y.cu = take(sizeof(float) * m);
    Y.Iulo = take(sizeof(float) * m);
    Y.Iuhi = take(sizeof(float) * m);
    Y.misc = take(sizeof(int) * 4);
    if (backward) {
        Y.vsnap = take(sizeof(float) * (N.L + 1) * (n + 1));
        size_t lv = 1, gl = (size_t)N.maxw * odd_ld(n);
        for (int l = 2; l <= N.L; ++l) {
            lv = std::max(lv, (size_t)lev_offset(N, l, l - 1));
            for (int k = 1; k <= l - (top_adjoint ? 1 : 2); ++k) gl = std::max(gl, (size_t)N.w[l] * odd_ld(N.w[k]));
        }
        Y.lev = take(sizeof(float) * lv);
        Y.gc = take(sizeof(double) * n);
        Y.gP = take(sizeof(double) * n * n);
        Y.gIlo = take(sizeof(double) * n);
        Y.gIhi = take(sizeof(double) * n);
        Y.gcn = take(sizeof(double) * n);
        Y.gPn = take(sizeof(double) * n * n);
        Y.gIlon = take(sizeof(double) * n);
        Y.gIhin = take(sizeof(double) * n);
        Y.gPu = take(sizeof(double) * m * n);
        Y.gcu = take(sizeof(double) * m);
        Y.gIulo = take(sizeof(double) * m);
        Y.gIuhi = take(sizeof(double) * m);
        Y.gv = take(sizeof(double) * n);
        Y.gw = take(sizeof(double) * 2);
        Y.gs = take(sizeof(float) * hid);
        Y.gd = take(sizeof(float) * hid);
        Y.gl = take(sizeof(float) * hid);
        Y.gu = take(sizeof(float) * hid);
        Y.gG = take(sizeof(float) * N.maxw * odd_ld(n));
        Y.ga = take(sizeof(float) * N.maxw);
        Y.gklo = take(sizeof(float) * N.maxw);
        Y.gkhi = take(sizeof(float) * N.maxw);
        Y.gRlo = take(sizeof(float) * N.maxw);
        Y.gRhi = take(sizeof(float) * N.maxw);
        Y.gL0 = take(sizeof(float) * gl);
        Y.gL1 = take(sizeof(float) * gl);
        if (((off + 15) & ~size_t(15)) > (size_t)kMaxSmem) {
            // slab mode anyway: keep every target's levels and kappa of the replayed step
            Y.levall = take(sizeof(float) * std::max(levall_offset(N, N.L + 1), 1));
            Y.kall = take(sizeof(float) * 2 * kall_total(N));
        }
    }
    Y.total = (int)((off + 15) & ~size_t(15));
    if (backward && !top_adjoint && Y.total > kMaxSmem) return fused_layout(N, true, true);
    return Y;
}

static MultiLayout multi_layout(const NetDesc& N, int G) {
    MultiLayout Y;
    memset(&Y, 0, sizeof(Y));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 15) & ~size_t(15);
        const size_t r = off;
        off += bytes;
        return (int)r;
    };
    const int n = N.n, m = N.m;
    for (int l = 0; l < N.L; ++l) Y.Ws[l] = take(sizeof(float) * N.w[l + 1] * odd_ld(N.w[l]));
    int nb = 0;
    for (int l = 0; l < N.L; ++l) nb += N.w[l + 1];
    Y.bs = take(sizeof(float) * nb);
    Y.A = take(sizeof(double) * n * n);
    Y.B = take(sizeof(double) * n * m);
    Y.e = take(sizeof(double) * n);
    {
        size_t chain = 4, bsz = 4, esz = 2;
        for (int l = 2; l <= N.L; ++l) {
            for (int mm = l - 1; mm >= 1; --mm) chain = std::max(chain, (size_t)G * N.w[l] * odd_ld(N.w[mm - 1]));
            if (N.w[l - 2] <= 16) {
                chain = std::max(chain, (size_t)N.w[l] * ru4(G * N.w[l - 2]));
                bsz = std::max(bsz, (size_t)N.w[l - 1] * ru4(G * N.w[l - 2]));
            }
            esz = std::max(esz, (size_t)N.w[l - 1] * G * 2);
        }
        Y.chA = take(sizeof(float) * chain);
        Y.chB = take(sizeof(float) * chain);
        Y.Bs = take(sizeof(float) * bsz);
        Y.E = take(sizeof(float) * esz);
    }
    Y.dom0 = (int)((off + 15) & ~size_t(15));
    size_t d = 0;
    auto dtake = [&](size_t bytes) {
        d = (d + 15) & ~size_t(15);
        const size_t r = d;
        d += bytes;
        return (int)r;
    };
    Y.c = dtake(sizeof(double) * n);
    Y.P = dtake(sizeof(double) * n * n);
    Y.Ilo = dtake(sizeof(double) * n);
    Y.Ihi = dtake(sizeof(double) * n);
    Y.v = dtake(sizeof(double) * n);
    Y.w = dtake(sizeof(double) * 2);
    Y.cn = dtake(sizeof(double) * n);
    Y.Pn = dtake(sizeof(double) * n * n);
    Y.Ilon = dtake(sizeof(double) * n);
    Y.Ihin = dtake(sizeof(double) * n);
    Y.red = dtake(sizeof(double) * (n + 1));
    Y.cf = dtake(sizeof(float) * n);
    Y.Pf = dtake(sizeof(float) * n * n);
    Y.Ilof = dtake(sizeof(float) * n);
    Y.Ihif = dtake(sizeof(float) * n);
    Y.vf = dtake(sizeof(float) * (n + 1));
    const int hid = std::max(N.hidden, 1);
    Y.hl = dtake(sizeof(float) * hid);
    Y.hu = dtake(sizeof(float) * hid);
    Y.hs = dtake(sizeof(float) * hid);
    Y.hd = dtake(sizeof(float) * hid);
    Y.klo = dtake(sizeof(float) * N.maxw);
    Y.khi = dtake(sizeof(float) * N.maxw);
    Y.G = dtake(sizeof(float) * N.maxw * odd_ld(n));
    Y.a = dtake(sizeof(float) * N.maxw);
    Y.Rlo = dtake(sizeof(float) * N.maxw);
    Y.Rhi = dtake(sizeof(float) * N.maxw);
    Y.S = dtake(sizeof(float) * N.maxw);
    Y.cu = dtake(sizeof(float) * m);
    Y.Iulo = dtake(sizeof(float) * m);
    Y.Iuhi = dtake(sizeof(float) * m);
    Y.misc = dtake(sizeof(int) * 4);
    Y.stride = (int)((d + 15) & ~size_t(15));
    Y.total = Y.dom0 + G * Y.stride;
    return Y;
}


// Shared-memory layout of the warp-per-domain kernel (two hidden layers), WPC warps per CTA.
static bool warp_applicable(const NetDesc& N) {
    return N.L == 3 && N.n <= kWarpNX && N.m <= kWarpNX && N.w[1] <= kWarpHMAX && N.w[2] <= kWarpHMAX;
}

static WarpLayout warp_layout(const NetDesc& N, int WPC, bool splits) {
    WarpLayout Y;
    memset(&Y, 0, sizeof(Y));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 15) & ~size_t(15);
        const size_t r = off;
        off += bytes;
        return (int)r;
    };
    const int n = N.n, m = N.m, H1 = N.w[1], H2 = N.w[2];
    Y.ld1 = odd_ld(n);
    Y.ld2 = odd_ld(H1);
    Y.W1 = take(sizeof(float) * H1 * Y.ld1);
    Y.W2 = take(sizeof(float) * H2 * Y.ld2);
    Y.W3 = take(sizeof(float) * m * H2);
    Y.bs = take(sizeof(float) * (H1 + H2 + m));
    Y.A = take(sizeof(double) * n * n);
    Y.B = take(sizeof(double) * n * m);
    Y.e = take(sizeof(double) * n);
    Y.dom0 = (int)((off + 15) & ~size_t(15));
    size_t d = 0;
    auto dtake = [&](size_t bytes) {
        d = (d + 15) & ~size_t(15);
        const size_t r = d;
        d += bytes;
        return (int)r;
    };
    Y.c = dtake(sizeof(double) * n);
    Y.P = dtake(sizeof(double) * n * n);
    Y.Ilo = dtake(sizeof(double) * n);
    Y.Ihi = dtake(sizeof(double) * n);
    Y.v = dtake(sizeof(double) * n);
    Y.w = dtake(sizeof(double) * 1);
    Y.cn = dtake(sizeof(double) * n);
    Y.Pn = dtake(sizeof(double) * n * n);
    Y.Ilon = dtake(sizeof(double) * n);
    Y.Ihin = dtake(sizeof(double) * n);
    Y.cf = dtake(sizeof(float) * n);
    Y.Pf = dtake(sizeof(float) * n * n);
    Y.Ilof = dtake(sizeof(float) * n);
    Y.Ihif = dtake(sizeof(float) * n);
    Y.vf = dtake(sizeof(float) * (n + 1));
    Y.hl = dtake(sizeof(float) * (H1 + H2));
    Y.hu = dtake(sizeof(float) * (H1 + H2));
    Y.hs = dtake(sizeof(float) * (H1 + H2));
    Y.hd = dtake(sizeof(float) * (H1 + H2));
    Y.sb1 = dtake(sizeof(float) * H1);
    Y.B1 = dtake(sizeof(float) * H1 * ((n + 3) & ~3));
    Y.W3s = dtake(sizeof(float) * m * H2);
    Y.L31 = dtake(sizeof(float) * m * H1);
    Y.Lx3 = dtake(sizeof(float) * m * n);
    Y.Pu = dtake(sizeof(float) * m * kWarpNX);
    Y.cu = dtake(sizeof(float) * m);
    Y.Iulo = dtake(sizeof(float) * m);
    Y.Iuhi = dtake(sizeof(float) * m);
    const int hm = splits ? std::max(H1, H2) : 1;
    Y.sa = dtake(sizeof(float) * hm);
    Y.klo = dtake(sizeof(float) * hm);
    Y.khi = dtake(sizeof(float) * hm);
    Y.sRlo = dtake(sizeof(float) * hm);
    Y.sRhi = dtake(sizeof(float) * hm);
    Y.sS = dtake(sizeof(float) * hm);
    Y.Gs = dtake(sizeof(float) * hm * kWarpNX);
    Y.misc = dtake(sizeof(int) * 4);
    Y.stride = (int)((d + 15) & ~size_t(15));
    Y.total = Y.dom0 + WPC * Y.stride;
    return Y;
}


static bool fused_fits(const NetDesc& N) { return fused_layout(N).total <= kMaxSmem; }

static int fused_threads(const NetDesc& N) { return N.maxw <= 64 ? 128 : 256; }

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------

// ------------------------------------------------------------------------------------------------
// tensor-core GEMM plumbing
// ------------------------------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static int get_encoder(dr_ctx* c) {
    if (g_encode) return DR_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(c, DR_ERR_CUDA, "cuTensorMapEncodeTiled unavailable (%s)", cudaGetErrorString(e));
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return DR_OK;
}

// 2D FP32 tensor map over rows x ldk (K contiguous), box 32 x box_rows, 128-byte swizzle.
static int make_map(dr_ctx* c, CUtensorMap* map, const float* ptr, int64_t rows, int ldk, int box_rows) {
    if ((reinterpret_cast<uintptr_t>(ptr) & 15) || (ldk % tc::BK)) return fail(c, DR_ERR_ARG, "tensor map alignment");
    cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ldk * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, DR_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return DR_OK;
}

// Tensor map over a blocked left operand (tc::blk_index) of R rows (padded to whole 128-row tiles)
// and ldk columns: a 2D view [tiles * ldk/32 * 128][32], box 32 x 128, 128-byte swizzle.
static int make_map_blocked(dr_ctx* c, CUtensorMap* map, const float* ptr, int64_t R, int ldk) {
    const int64_t rows = ((R + tc::BM - 1) / tc::BM) * (ldk / tc::BK) * tc::BM;
    if (rows > 0x7fffffffll) return fail(c, DR_ERR_SHAPE, "left operand too large for the tensor map (%lld rows)", (long long)R);
    return make_map(c, map, ptr, rows, tc::BK, tc::BM);
}

static int tc_bn(int N) { return N > 64 ? 128 : (N > 32 ? 64 : (N > 16 ? 32 : 16)); }

template <int BN, int EPI>
static int launch_tc_gemm_bn(dr_ctx* c, const CUtensorMap* m, float* C, int R, int K, int N, int ldc, int* err,
                             cudaStream_t st, const tc::ChainEpi& epi) {
    const int smem = tc::psmem_bytes(BN);
    CUDA_TRY(c, cudaFuncSetAttribute(tc::k_tc_gemm_p<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    // column tiles fastest: the CTAs sharing a row tile of A run together (one HBM read of A)
    const int64_t mt = (R + tc::BM - 1) / tc::BM;
    if (mt > 65535) return fail(c, DR_ERR_SHAPE, "too many row tiles (%lld) for one launch", (long long)mt);
    dim3 grid((N + BN - 1) / BN, (unsigned)mt);
    tc::k_tc_gemm_p<BN, EPI><<<grid, tc::gemm_threads(BN), smem, st>>>(m[0], m[1], m[2], m[3], m[4], m[5], C, R, K, N, ldc, err, epi);
    CUDA_TRY(c, cudaGetLastError());
    if (c) c->launches++;
    return DR_OK;
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 0;
        if (n <= 0) n = 1;
    }
    return n;
}

// The persistent kernel's warpgroup register split needs exactly the registers it was designed for
// at entry; a build that compiled it otherwise keeps the one-tile-per-CTA kernel.
template <int EPI, bool PAIR = false>
static bool persistent_gemm_usable() {
    static int ok = -1;
    if (ok < 0) {
        cudaFuncAttributes fa;
        ok = cudaFuncGetAttributes(&fa, tc::k_tc_gemm_pp<EPI, PAIR>) == cudaSuccess && fa.numRegs == tc::kRegsLaunch;
        cudaGetLastError();
    }
    return ok == 1;
}

// 128-column GEMMs with at least two tiles per SM run persistently (one CTA per SM, the epilogue of
// one tile overlapped with the main loop of the next).
// Clusters of `cs` CTAs (1 or 2): the CTAs of a cluster share the right operand's tile through a TMA
// multicast (tc_gemm_persistent.cuh).  The grid is at most the co-resident clusters (queried once per
// epilogue kind), so the kernel stays persistent.
template <int EPI, bool PAIR = false>
static int launch_tc_gemm_persistent(dr_ctx* c, const CUtensorMap* m, float* C, int R, int K, int N, int ldc, int* err,
                                     cudaStream_t st, const tc::ChainEpi& epi, int64_t tiles, int nsm, int cs = 2) {
    const int smem = tc::pp_smem_bytes();
    CUDA_TRY(c, cudaFuncSetAttribute(tc::k_tc_gemm_pp<EPI, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    if (PAIR) cs = 2;
    static int max_clusters = 0;  // co-resident clusters of two (-1: none)
    if (cs == 2 && max_clusters == 0) {
        if (c && c->capturing) {
            cs = 1;  // never queried outside a capture: no query inside one
        } else {
            cudaLaunchConfig_t q = {};
            q.gridDim = dim3((unsigned)(nsm & ~1));
            q.blockDim = dim3(tc::kPersistThreads);
            q.dynamicSmemBytes = smem;
            cudaLaunchAttribute qa[1];
            qa[0].id = cudaLaunchAttributeClusterDimension;
            qa[0].val.clusterDim.x = 2;
            qa[0].val.clusterDim.y = 1;
            qa[0].val.clusterDim.z = 1;
            q.attrs = qa;
            q.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, tc::k_tc_gemm_pp<EPI, PAIR>, &q) != cudaSuccess || n < 1) n = -1;
            cudaGetLastError();
            max_clusters = n;
        }
    }
    if (PAIR && max_clusters < 1) return fail(c, DR_ERR_STATE, "the pair GEMM needs clusters of two CTAs");
    if (cs == 2 && max_clusters < 1) cs = 1;  // no cluster launch here: every CTA loads both operands
    const int64_t mtn = (R + tc::BM - 1) / tc::BM, ntn = (N + 127) / 128;
    const int64_t ctiles = ((mtn + cs - 1) / cs) * ntn;
    int64_t nclu = std::min<int64_t>(ctiles, cs == 2 ? max_clusters : nsm);
    if (nclu < 1) nclu = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclu * cs));
    cfg.blockDim = dim3(tc::kPersistThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CUDA_TRY(c, cudaLaunchKernelEx(&cfg, tc::k_tc_gemm_pp<EPI, PAIR>, m[0], m[1], m[2], m[3], C, R, K, N, ldc, err, epi));
    if (c) c->launches++;
    (void)tiles;
    return DR_OK;
}

// Launch shapes of the tensor-core GEMM (dr_options.tuning = 0 picks one per shape by timing them):
// 0 = the heuristic (the persistent kernel for 128-column tiles with at least two tiles per SM, else
// one 128 x tc_bn(N) tile per CTA), 1 = persistent 128 x 128 in clusters of two CTAs sharing the
// right operand's tiles, 2 = one 128 x 128 tile per CTA, 3 = one 128 x 64 tile per CTA, 4 = one
// 128 x 32 tile per CTA, 5 = persistent 128 x 128 without clusters, 6 = persistent pair form (one
// cta_group::2 MMA of M = 256 over a CTA pair, B's columns split between the two CTAs).
enum { kGemmHeuristic = 0, kGemmPersistent = 1, kGemmTile128 = 2, kGemmTile64 = 3, kGemmTile32 = 4, kGemmPersistent1 = 5, kGemmPair = 6 };

static int tc_gemm_launch(dr_ctx* c, const float* Ah, const float* Al, const float* BTh, const float* BTl, float* C, int R,
                          int K, int N, int ldk, int ldc, int* err, cudaStream_t st, const tc::ChainEpi* epi, int* cls,
                          int variant, int* bn_used);

static cudaEvent_t kt_event(dr_ctx* c) {
    cudaEvent_t e = nullptr;
    if (!c->kt_pool.empty()) {
        e = c->kt_pool.back();
        c->kt_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        e = nullptr;
    }
    return e;
}

// Autotuner of the tensor-core GEMM's launch shape: the first time a shape (epilogue kind, R, K, N,
// SM count) is met outside a graph capture, every candidate runs twice on the real operands (each
// run writes the same outputs from the same inputs) and the second run is timed with CUDA events;
// the fastest is cached for the process and, if it was not the last one run, runs once more so that
// the outputs are its own.  Captured and later calls reuse the cached choice; an uncached shape met
// while capturing takes the heuristic.
static std::mutex g_gemm_mu;
static std::map<std::string, int> g_gemm_choice;
static std::map<std::string, std::string> g_gemm_report;

static std::string gemm_key(const tc::ChainEpi* epi, int R, int K, int N) {
    char buf[96];
    snprintf(buf, sizeof(buf), "epi%d R%d K%d N%d sm%d", !epi ? 0 : (epi->W1 ? 2 : 1), R, K, N, sm_count());
    return buf;
}

// GEMM tuning cache file (optional, path from DR_GEMM_TUNE_CACHE): one "key variant" pair per line,
// the key's spaces written as '_'.  Choices in the file are taken as they are (no trials); new
// choices are appended to the map and the whole map is written back.  A profiler run of the same
// program then launches the shapes the plain run picked (under a profiler the trials' timings are
// distorted).  Called with g_gemm_mu held.
static bool g_gemm_file_loaded = false;
static void gemm_file_load() {
    if (g_gemm_file_loaded) return;
    g_gemm_file_loaded = true;
    const char* path = getenv("DR_GEMM_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[256];
    int v;
    while (fscanf(f, "%255s %d", key, &v) == 2) {
        if (v < kGemmPersistent || v > kGemmPair) continue;
        std::string k(key);
        std::replace(k.begin(), k.end(), '_', ' ');
        g_gemm_choice[k] = v;
        g_gemm_report[k] = "variant " + std::to_string(v) + " (from DR_GEMM_TUNE_CACHE)";
    }
    fclose(f);
}
static void gemm_file_store() {
    const char* path = getenv("DR_GEMM_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    for (const auto& kv : g_gemm_choice) {
        std::string k = kv.first;
        std::replace(k.begin(), k.end(), ' ', '_');
        fprintf(f, "%s %d\n", k.c_str(), kv.second);
    }
    fclose(f);
}

static int tuned_gemm(dr_ctx* c, const float* Ah, const float* Al, const float* BTh, const float* BTl, float* C, int R, int K,
                      int N, int ldk, int ldc, int* err, cudaStream_t st, const tc::ChainEpi* epi, int* variant) {
    const std::string key = gemm_key(epi, R, K, N);
    {
        std::lock_guard<std::mutex> lock(g_gemm_mu);
        gemm_file_load();
        auto it = g_gemm_choice.find(key);
        if (it != g_gemm_choice.end()) {
            *variant = it->second;
            return DR_OK;
        }
    }
    if (c->capturing) return DR_OK;  // heuristic
    int cand[6], nc = 0;
    if (tc_bn(N) == 128) {
        if (persistent_gemm_usable<0>() && persistent_gemm_usable<1>() && persistent_gemm_usable<2>()) {
            cand[nc++] = kGemmPersistent;
            cand[nc++] = kGemmPersistent1;
        }
        if (persistent_gemm_usable<0, true>() && persistent_gemm_usable<1, true>() && persistent_gemm_usable<2, true>())
            cand[nc++] = kGemmPair;
        cand[nc++] = kGemmTile128;
    }
    if (N > 32) cand[nc++] = kGemmTile64;
    if (N > 16 && N <= 64) cand[nc++] = kGemmTile32;
    if (nc <= 1) {
        *variant = nc ? cand[0] : kGemmHeuristic;
        return DR_OK;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, DR_ERR_CUDA, "cudaEventCreate");
    }
    float best = 0.f, ms[6] = {};
    int pick = cand[0], rc = DR_OK;
    for (int q = 0; q < nc && rc == DR_OK; ++q) {
        for (int rep = 0; rep < 2 && rc == DR_OK; ++rep) {
            int cls = 0, bn = 0;
            if (cudaEventRecord(e0, st) != cudaSuccess) rc = fail(c, DR_ERR_CUDA, "cudaEventRecord");
            if (rc == DR_OK) rc = tc_gemm_launch(c, Ah, Al, BTh, BTl, C, R, K, N, ldk, ldc, err, st, epi, &cls, cand[q], &bn);
            if (rc == DR_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&ms[q], e0, e1) != cudaSuccess))
                rc = fail(c, DR_ERR_CUDA, "GEMM tuning: %s", cudaGetErrorString(cudaGetLastError()));
        }
        if (rc == DR_OK && (q == 0 || ms[q] < best)) {
            best = ms[q];
            pick = cand[q];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TRY(rc);
    int herr = 0;  // a bounded pipeline wait that expired during the trials
    CUDA_TRY(c, cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return fail(c, DR_ERR_TIMEOUT, "a tensor-core pipeline wait timed out while tuning");
    {
        std::lock_guard<std::mutex> lock(g_gemm_mu);
        g_gemm_choice[key] = pick;
        std::string rep = "variant " + std::to_string(pick) + " (ms:";
        for (int q = 0; q < nc; ++q) {
            char b[48];
            snprintf(b, sizeof(b), " v%d=%.3f", cand[q], ms[q]);
            rep += b;
        }
        g_gemm_report[key] = rep + ")";
        gemm_file_store();
    }
    *variant = pick;  // the caller then launches the pick, so the outputs are its own
    return DR_OK;
}

// C [R x N] (ld ldc) = A B with A given as TF32 parts Ah/Al (blocked layout, tc::blk_index, ldk
// columns) and B as BTh/BTl [N][ldk]; with `epi` the chain epilogue replaces the store of C.  With
// dr_options.timing set (and not capturing a graph) the launch is bracketed by two CUDA events on `st`.
static int tc_gemm(dr_ctx* c, const float* Ah, const float* Al, const float* BTh, const float* BTl, float* C, int R, int K,
                   int N, int ldk, int ldc, int* err, cudaStream_t st, const tc::ChainEpi* epi = nullptr, int* bn_used = nullptr) {
    int bn_dummy = 0;
    if (!bn_used) bn_used = &bn_dummy;
    int variant = kGemmHeuristic;
    if (c && c->opt.tuning == 0 && !(epi && epi->colpart)) TRY(tuned_gemm(c, Ah, Al, BTh, BTl, C, R, K, N, ldk, ldc, err, st, epi, &variant));
    if (c && c->opt.tuning >= 100) variant = c->opt.tuning - 100;  // forced launch shape
    const bool timed = c && c->opt.timing && !c->capturing;
    cudaEvent_t e0 = timed ? kt_event(c) : nullptr, e1 = timed ? kt_event(c) : nullptr;
    if (e0 && e1) CUDA_TRY(c, cudaEventRecord(e0, st));
    int cls = DR_KT_GEMM_OTHER;
    const int rc = tc_gemm_launch(c, Ah, Al, BTh, BTl, C, R, K, N, ldk, ldc, err, st, epi, &cls, variant, bn_used);
    if (timed) {
        if (rc == DR_OK && e0 && e1) {
            CUDA_TRY(c, cudaEventRecord(e1, st));
            double flop = 2.0 * R * K * N;
            if (epi && epi->W1) flop += 2.0 * R * N * epi->n0;
            c->kt_pending.push_back({cls, (int64_t)R, e0, e1, flop});
        } else {
            if (e0) c->kt_pool.push_back(e0);
            if (e1) c->kt_pool.push_back(e1);
        }
    }
    return rc;
}

static int tc_gemm_launch(dr_ctx* c, const float* Ah, const float* Al, const float* BTh, const float* BTl, float* C, int R,
                          int K, int N, int ldk, int ldc, int* err, cudaStream_t st, const tc::ChainEpi* epi, int* cls,
                          int variant, int* bn_used) {
    TRY(get_encoder(c));
    // the reverse chain level runs only on the persistent kernel, whose stages hold 128-row B boxes
    const int BN = (epi && epi->colpart) ? 128
                   : variant == kGemmTile64 ? 64 : variant == kGemmTile32 ? 32 : variant >= kGemmPersistent ? 128 : tc_bn(N);
    const int ccs = variant == kGemmPersistent1 ? 1 : 2;  // cluster size of a persistent launch
    *bn_used = BN;
    CUtensorMap m[6];
    TRY(make_map_blocked(c, &m[0], Ah, R, ldk));
    TRY(make_map_blocked(c, &m[1], Al, R, ldk));
    const bool pair = variant == kGemmPair && !(epi && epi->colpart);
    TRY(make_map(c, &m[2], BTh, N, ldk, pair ? BN / 2 : BN));  // the pair form: each CTA loads half of B's columns
    TRY(make_map(c, &m[3], BTl, N, ldk, pair ? BN / 2 : BN));
    if (epi && epi->colpart) {
        m[4] = m[0];
        m[5] = m[1];
    } else if (epi && !epi->W1) {
        // the chain epilogue stores the next left operand (blocked, epi->ldk columns) by TMA
        TRY(make_map_blocked(c, &m[4], epi->Ah, R, epi->ldk));
        TRY(make_map_blocked(c, &m[5], epi->Al, R, epi->ldk));
    } else {
        m[4] = m[0];
        m[5] = m[1];
    }
    tc::ChainEpi e{};
    if (epi) e = *epi;
    if (epi && epi->W1 && (BN < 32 || epi->n0 > tc::kFinalCols))
        return fail(c, DR_ERR_SHAPE, "fused final chain level needs >= 32 columns and n <= %d", tc::kFinalCols);
    if (epi && epi->colpart) {
        // reverse chain level: the persistent kernel's reverse epilogue (the only launch shape)
        if (!persistent_gemm_usable<3>()) return fail(c, DR_ERR_STATE, "the reverse chain GEMM is unavailable in this build");
        const int64_t tiles = ((int64_t)(R + tc::BM - 1) / tc::BM) * ((N + 127) / 128);
        if (tiles > 0x7fffffffll) return fail(c, DR_ERR_SHAPE, "too many tiles for one reverse GEMM");
        *bn_used = 128;
        *cls = DR_KT_GEMM_REVERSE;
        return launch_tc_gemm_persistent<3>(c, m, C, R, K, N, ldc, err, st, e, tiles, sm_count(), ccs);
    }
    if (BN == 128 && variant != kGemmTile128) {
        const int nsm = sm_count();
        const int64_t tiles = ((int64_t)(R + tc::BM - 1) / tc::BM) * ((N + 127) / 128);
        if (pair && tiles <= 0x7fffffffll) {
            if (!epi) return launch_tc_gemm_persistent<0, true>(c, m, C, R, K, N, ldc, err, st, e, tiles, nsm);
            if (epi->W1) {
                *cls = DR_KT_GEMM_FINAL;
                return launch_tc_gemm_persistent<2, true>(c, m, C, R, K, N, ldc, err, st, e, tiles, nsm);
            }
            *cls = DR_KT_GEMM_CHAIN;
            return launch_tc_gemm_persistent<1, true>(c, m, C, R, K, N, ldc, err, st, e, tiles, nsm);
        }
        if ((variant == kGemmPersistent || variant == kGemmPersistent1 || tiles >= 2 * (int64_t)nsm) && tiles <= 0x7fffffffll) {
            if (!epi && persistent_gemm_usable<0>())
                return launch_tc_gemm_persistent<0>(c, m, C, R, K, N, ldc, err, st, e, tiles, nsm, ccs);
            if (epi && epi->W1 && persistent_gemm_usable<2>()) {
                *cls = DR_KT_GEMM_FINAL;
                return launch_tc_gemm_persistent<2>(c, m, C, R, K, N, ldc, err, st, e, tiles, nsm, ccs);
            }
            if (epi && !epi->W1 && persistent_gemm_usable<1>()) {
                *cls = DR_KT_GEMM_CHAIN;
                return launch_tc_gemm_persistent<1>(c, m, C, R, K, N, ldc, err, st, e, tiles, nsm, ccs);
            }
        }
    }
#define DR_TC_CASE(bn)                                                                                        \
    case bn:                                                                                                  \
        return !epi ? launch_tc_gemm_bn<bn, 0>(c, m, C, R, K, N, ldc, err, st, e)                             \
                    : (epi->W1 ? launch_tc_gemm_bn<bn, 2>(c, m, C, R, K, N, ldc, err, st, e)                  \
                               : launch_tc_gemm_bn<bn, 1>(c, m, C, R, K, N, ldc, err, st, e));
    switch (BN) {
        DR_TC_CASE(128)
        DR_TC_CASE(64)
        DR_TC_CASE(32)
        default:
            return epi ? launch_tc_gemm_bn<16, 1>(c, m, C, R, K, N, ldc, err, st, e)
                       : launch_tc_gemm_bn<16, 0>(c, m, C, R, K, N, ldc, err, st, e);
    }
#undef DR_TC_CASE
}

static inline int round_up32(int x) { return (x + 31) & ~31; }

// ------------------------------------------------------------------------------------------------
// grouped fused kernel: launch variants and the autotuner
// ------------------------------------------------------------------------------------------------

// Launch variants of the bounds-only forward pass: warp-per-domain kernels (group < 0: -group
// warps per CTA; controllers with two hidden layers) and grouped kernels (threads, domains per CTA).
struct MultiVariant {
    int threads, group;
};
static const MultiVariant kMultiVariants[] = {{512, -16}, {256, -8}, {128, -4}, {256, 8}, {512, 8}, {256, 4},
                                              {512, 4},   {128, 2},  {256, 2},  {128, 1}};
static const int kNumMultiVariants = (int)(sizeof(kMultiVariants) / sizeof(kMultiVariants[0]));

static bool variant_fits(const MultiArgs& a, int v) {
    const MultiVariant mv = kMultiVariants[v];
    if (mv.group < 0)
        return warp_applicable(a.net) && warp_layout(a.net, -mv.group, a.sp_row != nullptr).total <= kMaxSmem;
    return multi_layout(a.net, mv.group).total <= kMaxSmem;
}

template <int WPC>
static int launch_warp_t(dr_ctx* c, const MultiArgs& a) {
    const bool splits = a.sp_row != nullptr;
    const WarpLayout Y = warp_layout(a.net, WPC, splits);
    if (!warp_applicable(a.net) || Y.total > kMaxSmem) return fail(c, DR_ERR_SHAPE, "warp variant does not fit");
    CUDA_TRY(c, cudaFuncSetAttribute(k_fused_warp<WPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, Y.total));
    k_fused_warp<WPC><<<(unsigned)((a.D + WPC - 1) / WPC), 32 * WPC, Y.total, c->stream>>>(a, Y, splits ? 1 : 0);
    CUDA_TRY(c, cudaGetLastError());
    c->launches++;
    return DR_OK;
}

template <int NT, int G>
static int launch_multi_t(dr_ctx* c, MultiArgs a) {
    a.lay = multi_layout(a.net, G);
    const int smem = a.lay.total;
    if (smem > kMaxSmem) return fail(c, DR_ERR_SHAPE, "grouped variant does not fit shared memory");
    CUDA_TRY(c, cudaFuncSetAttribute(k_fused_forward_multi<NT, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_fused_forward_multi<NT, G><<<(unsigned)((a.D + G - 1) / G), NT, smem, c->stream>>>(a);
    CUDA_TRY(c, cudaGetLastError());
    c->launches++;
    return DR_OK;
}

static int launch_multi(dr_ctx* c, const MultiArgs& a, int v) {
    switch (v) {
        case 0: return launch_warp_t<16>(c, a);
        case 1: return launch_warp_t<8>(c, a);
        case 2: return launch_warp_t<4>(c, a);
        case 3: return launch_multi_t<256, 8>(c, a);
        case 4: return launch_multi_t<512, 8>(c, a);
        case 5: return launch_multi_t<256, 4>(c, a);
        case 6: return launch_multi_t<512, 4>(c, a);
        case 7: return launch_multi_t<128, 2>(c, a);
        case 8: return launch_multi_t<256, 2>(c, a);
        default: return launch_multi_t<128, 1>(c, a);
    }
}

static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;
static bool g_tune_file_loaded = false;

static std::string tune_key(const NetDesc& N, int dev) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    std::string k = std::string("sm") + std::to_string(prop.major) + std::to_string(prop.minor) + ":";
    for (int l = 0; l <= N.L; ++l) k += std::to_string(N.w[l]) + (l < N.L ? "-" : "");
    return k;
}

// Tuning cache file (optional): one "key variant" pair per line, path from DR_TUNE_CACHE.
static void tune_file_load() {
    if (g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    const char* path = getenv("DR_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[512];
    int v;
    while (fscanf(f, "%511s %d", key, &v) == 2)
        if (v >= 0 && v < kNumMultiVariants) g_tune_cache[key] = v;
    fclose(f);
}

static void tune_file_store() {
    const char* path = getenv("DR_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    for (const auto& kv : g_tune_cache) fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
    fclose(f);
}

// Pick the fastest fitting (threads, domains per CTA) variant for this controller shape: each
// candidate runs once untimed and twice timed (the better time counts) on the first 16,384 domains
// (all of them when fewer) and 2 steps (CUDA events on the context's stream), the winner is cached
// per (architecture, widths).  dr_options.tuning = 1 disables the
// search and takes the first fitting variant with the largest group.
static int tuned_variant(dr_ctx* c, const MultiArgs& a, int* out) {
    if (c->opt.tuning >= 2 && c->opt.tuning < 100) {
        const int v = c->opt.tuning - 2;
        if (v >= kNumMultiVariants || !variant_fits(a, v))
            return fail(c, DR_ERR_SHAPE, "launch variant %d does not fit this controller", v);
        *out = v;
        return DR_OK;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_file_load();
    const std::string key = tune_key(a.net, c->device) + (a.sp_row ? ":splits" : "");
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
        *out = it->second;
        return DR_OK;
    }
    int first_fit = -1;
    for (int v = 0; v < kNumMultiVariants; ++v)
        if (variant_fits(a, v)) {
            first_fit = v;
            break;
        }
    if (first_fit < 0) return fail(c, DR_ERR_SHAPE, "no grouped variant fits shared memory");
    if (c->opt.tuning == 1 || c->opt.tuning >= 100 || c->D == 0) {
        *out = first_fit;
        return DR_OK;
    }
    MultiArgs t = a;
    // the real launch's grid (its wave pattern decides between variants whose times differ by a few
    // per cent) up to 16,384 domains, two steps
    t.D = std::min<int64_t>(a.D, 16384);
    t.net.H = std::min(a.net.H, 2);
    t.V = nullptr;
    t.status = nullptr;
    t.alpha_used = nullptr;
    cudaEvent_t e0, e1;
    CUDA_TRY(c, cudaEventCreate(&e0));
    CUDA_TRY(c, cudaEventCreate(&e1));
    float best = 1e30f;
    int bestv = first_fit;
    for (int v = 0; v < kNumMultiVariants; ++v) {
        if (!variant_fits(a, v)) continue;
        TRY(launch_multi(c, t, v));  // warm-up
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {  // the better of two timed runs
            CUDA_TRY(c, cudaEventRecord(e0, c->stream));
            TRY(launch_multi(c, t, v));
            CUDA_TRY(c, cudaEventRecord(e1, c->stream));
            CUDA_TRY(c, cudaEventSynchronize(e1));
            float r = 0.f;
            CUDA_TRY(c, cudaEventElapsedTime(&r, e0, e1));
            ms = std::min(ms, r);
        }
        if (ms < best) {
            best = ms;
            bestv = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_tune_cache[key] = bestv;
    tune_file_store();
    *out = bestv;
    return DR_OK;
}

extern "C" {

int dr_create(dr_ctx** out, int device, void* cuda_stream) {
    if (!out) return fail(nullptr, DR_ERR_ARG, "dr_create: out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count <= device || device < 0)
        return fail(nullptr, DR_ERR_CUDA, "dr_create: no CUDA device %d (%s)", device,
                    e == cudaSuccess ? "not present" : cudaGetErrorString(e));
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return fail(nullptr, DR_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    if (prop.major != 10 || prop.minor != 3)
        return fail(nullptr, DR_ERR_CUDA, "dr_create: device %d is sm_%d%d, this library is built for sm_103a", device,
                    prop.major, prop.minor);
    dr_ctx* c = new dr_ctx();
    c->device = device;
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    c->opt = default_options();
    *out = c;
    return DR_OK;
}

static void free_outputs(dr_ctx* c) {
    const size_t ob = c->out_bytes;
    dev_free(c, (void*&)c->dout_lo, ob);
    dev_free(c, (void*&)c->dout_hi, ob);
    dev_free(c, (void*&)c->dV, sizeof(double) * c->D);
    dev_free(c, (void*&)c->dstatus, sizeof(uint32_t) * c->D);
    dev_free(c, (void*&)c->dhull, sizeof(double) * 2 * (c->H + 1) * std::max(c->net.n, 1));
    dev_free(c, (void*&)c->dtape, c->tape_bytes);
    dev_free(c, (void*&)c->dgalpha, 0);
    dev_free(c, (void*&)c->dgbeta, 0);
    dev_free(c, (void*&)c->dbest_alpha, 0);
    dev_free(c, (void*&)c->dbest_beta, 0);
    dev_free(c, (void*&)c->dbestV, 0);
    dev_free(c, (void*&)c->dVhist, 0);
    dev_free(c, (void*&)c->dhist_slot, 0);
    dev_free(c, (void*&)c->dwlo, 0);
    dev_free(c, (void*&)c->dwhi, 0);
    dev_free(c, (void*&)c->dgshift, 0);
    c->gshift_valid = false;
    dev_free(c, (void*&)c->dgth, c->gth_bytes);
    c->gth_bytes = 0;
    dev_free(c, (void*&)c->dgth_part, 0);
    dev_free(c, (void*&)c->dgtheta, 0);
    c->gtheta_valid = false;
    dev_free(c, c->wscratch, c->wscratch_bytes);
    c->wscratch_bytes = 0;
    dev_free(c, (void*&)c->gslab, c->gslab_bytes);
    c->gslab_bytes = 0;
    dev_free(c, (void*&)c->dWpad, 0);
    dev_free(c, c->kscratch, c->kscratch_bytes);
    c->kscratch_bytes = 0;
    dev_free(c, (void*&)c->dsph, 0);
    c->wDc = 0;
    c->out_bytes = 0;
    c->tape_bytes = 0;
}

void dr_destroy(dr_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_outputs(c);
    cudaFree(c->dW);
    cudaFree(c->db);
    cudaFree(c->dA);
    cudaFree(c->dB);
    cudaFree(c->de);
    cudaFree(c->dlo0);
    cudaFree(c->dhi0);
    cudaFree(c->dsp_row);
    cudaFree(c->dsp);
    cudaFree(c->dbeta);
    cudaFree(c->dalpha);
    cudaFree(c->deoff);
    cudaFree(c->dWTh);
    cudaFree(c->dWTl);
    cudaFree(c->dA2h);
    cudaFree(c->dA2l);
    cudaFree(c->dA2ph);
    cudaFree(c->dA2pl);
    cudaFree(c->dWRh);
    cudaFree(c->dWRl);
    cudaFree(c->dWlev);
    cudaFree(c->derr);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (int l = 0; l < dr_ctx::kMaxLanes; ++l) {
        if (c->aux[l]) cudaStreamDestroy(c->aux[l]);
        if (c->ev_join[l]) cudaEventDestroy(c->ev_join[l]);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    for (auto& p : c->kt_pending) {
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
    }
    for (cudaEvent_t e : c->kt_pool) cudaEventDestroy(e);
    delete c;
}

const char* dr_last_error(const dr_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

int64_t dr_kernel_launches(const dr_ctx* c) { return c ? c->launches : 0; }

int64_t dr_graph_replays(const dr_ctx* c) { return c ? c->graph_replays : 0; }

int64_t dr_gemm_tuning_report(char* buf, int64_t cap) {
    std::string out;
    {
        std::lock_guard<std::mutex> lock(g_gemm_mu);
        for (const auto& kv : g_gemm_report) out += kv.first + ": " + kv.second + "\n";
    }
    if (buf && cap > 0) {
        const int64_t k = std::min<int64_t>(cap - 1, (int64_t)out.size());
        memcpy(buf, out.data(), (size_t)k);
        buf[k] = 0;
    }
    return (int64_t)out.size() + 1;
}

int dr_set_options(dr_ctx* c, const dr_options* o) {
    if (!c) return DR_ERR_ARG;
    dr_options n = o ? *o : default_options();
    if (n.slope_mode < 0 || n.slope_mode > 3) return fail(c, DR_ERR_ARG, "slope_mode %d out of range", n.slope_mode);
    if (n.precision < 0 || n.precision > 2) return fail(c, DR_ERR_ARG, "precision %d out of range", n.precision);
    if (!(n.margin_rho >= 0.0) || n.margin_rho > 1e-2) return fail(c, DR_ERR_ARG, "margin_rho %g out of range", n.margin_rho);
    if (!(n.box_margin >= 0.0) || n.box_margin > 1e-2) return fail(c, DR_ERR_ARG, "box_margin %g out of range", n.box_margin);
    if (n.chunk_domains < 0 || n.mem_cap_bytes < 0) return fail(c, DR_ERR_ARG, "negative chunk or memory cap");
    if (n.slope_mode == DR_SLOPE_USER && !c->alpha_set && c->D > 0)
        return fail(c, DR_ERR_STATE, "DR_SLOPE_USER requires dr_set_alpha first");
    if (n.timing < 0 || n.timing > 1) return fail(c, DR_ERR_ARG, "timing %d out of range", n.timing);
    if (n.rigorous < 0 || n.rigorous > 1) return fail(c, DR_ERR_ARG, "rigorous %d out of range", n.rigorous);
    if (n.weight_grad < 0 || n.weight_grad > 1) return fail(c, DR_ERR_ARG, "weight_grad %d out of range", n.weight_grad);
    if (n.reverse < 0 || n.reverse > 2) return fail(c, DR_ERR_ARG, "reverse %d out of range", n.reverse);
    if (n.tuning < 0 || (n.tuning >= 2 + kNumMultiVariants && (n.tuning < 101 || n.tuning > 106)))
        return fail(c, DR_ERR_ARG, "tuning %d out of range", n.tuning);
    if (n.timing && !c->opt.timing) c->kt_done.clear();  // timing switched on: the totals start from zero
    c->opt = n;
    c->epoch++;  // kernel arguments may change
    return DR_OK;
}

// Read the recorded event pairs into the per-class totals (waits for them) and recycle the events.
static int kt_drain(dr_ctx* c) {
    int rc = DR_OK;
    for (auto& p : c->kt_pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(p.e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.e0, p.e1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(c, DR_ERR_CUDA, "dr_kernel_timing: %s", cudaGetErrorString(e));
        } else {
            c->kt_done.push_back({p.cls, p.rows, (double)ms, p.flop});
        }
        c->kt_pool.push_back(p.e0);
        c->kt_pool.push_back(p.e1);
    }
    c->kt_pending.clear();
    return rc;
}

int dr_kernel_timing(dr_ctx* c, int which, int64_t min_rows, int64_t* launches, double* ms, double* flop) {
    if (!c) return DR_ERR_ARG;
    if (which < DR_KT_GEMM_ALL || which > DR_KT_GEMM_REVERSE) return fail(c, DR_ERR_ARG, "timing class %d", which);
    CUDA_TRY(c, cudaSetDevice(c->device));
    TRY(kt_drain(c));
    int64_t n = 0;
    double t = 0.0, f = 0.0;
    for (const auto& d : c->kt_done) {
        if ((which != DR_KT_GEMM_ALL && which != d.cls) || d.rows < min_rows) continue;
        n++;
        t += d.ms;
        f += d.flop;
    }
    if (launches) *launches = n;
    if (ms) *ms = t;
    if (flop) *flop = f;
    return DR_OK;
}

int dr_load_controller(dr_ctx* c, int L, const int32_t* widths, const void* const* W, const void* const* b, int dtype) {
    if (!c || !widths || !W || !b) return fail(c, DR_ERR_ARG, "dr_load_controller: NULL argument");
    if (L < 1 || L > DR_MAXL) return fail(c, DR_ERR_SHAPE, "L = %d outside 1..%d", L, DR_MAXL);
    if (dtype != DR_F32 && dtype != DR_F64) return fail(c, DR_ERR_ARG, "dtype %d", dtype);
    if (c->has_dyn && (widths[0] != c->net.n || widths[L] != c->net.m))
        return fail(c, DR_ERR_SHAPE, "controller widths (%d..%d) do not match dynamics (n=%d, m=%d)", widths[0],
                    widths[L], c->net.n, c->net.m);
    NetDesc N{};
    N.L = L;
    int64_t nw = 0, nb = 0;
    N.maxw = 0;
    for (int l = 0; l <= L; ++l) {
        if (widths[l] < 1 || widths[l] > 4096) return fail(c, DR_ERR_SHAPE, "width[%d] = %d", l, widths[l]);
        N.w[l] = widths[l];
        if (l >= 1) N.maxw = std::max(N.maxw, widths[l]);
    }
    N.hidden = 0;
    for (int l = 1; l < L; ++l) {
        N.hoff[l] = N.hidden;
        N.hidden += widths[l];
    }
    N.hoff[L] = N.hidden;
    for (int l = 0; l < L; ++l) {
        N.Woff[l] = nw;
        N.boff[l] = nb;
        nw += (int64_t)widths[l + 1] * widths[l];
        nb += widths[l + 1];
    }
    N.n = widths[0];
    N.m = widths[L];
    N.H = c->H;
    std::vector<float> hw(nw), hb(nb);
    for (int l = 0; l < L; ++l) {
        const int64_t cnt = (int64_t)widths[l + 1] * widths[l];
        for (int64_t i = 0; i < cnt; ++i) {
            const double x = dtype == DR_F64 ? ((const double*)W[l])[i] : ((const float*)W[l])[i];
            if (!std::isfinite(x)) return fail(c, DR_ERR_NONFINITE, "non-finite weight in layer %d", l + 1);
            hw[N.Woff[l] + i] = (float)x;
        }
        for (int i = 0; i < widths[l + 1]; ++i) {
            const double x = dtype == DR_F64 ? ((const double*)b[l])[i] : ((const float*)b[l])[i];
            if (!std::isfinite(x)) return fail(c, DR_ERR_NONFINITE, "non-finite bias in layer %d", l + 1);
            hb[N.boff[l] + i] = (float)x;
        }
    }
    CUDA_TRY(c, cudaSetDevice(c->device));
    dev_free(c, (void*&)c->dW, 0);
    dev_free(c, (void*&)c->db, 0);
    dev_free(c, (void*&)c->dWpad, 0);
    TRY(dev_alloc(c, c->dW, nw));
    TRY(dev_alloc(c, c->db, nb));
    c->gshift_valid = false;  // gradients of the previous controller
    c->gtheta_valid = false;
    CUDA_TRY(c, cudaMemcpyAsync(c->dW, hw.data(), nw * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->db, hb.data(), nb * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    // transposed TF32 parts (round to nearest, ties away) for the tensor-core chain
    {
        auto tf32 = [](float x) {
            uint32_t u;
            memcpy(&u, &x, 4);
            if ((u & 0x7f800000u) != 0x7f800000u) {
                u += 0x1000u;
                u &= 0xffffe000u;
            }
            float r;
            memcpy(&r, &u, 4);
            return r;
        };
        int64_t tot = 0;
        int64_t offs[DR_MAXL];
        for (int l = 0; l < L; ++l) {
            offs[l] = tot;
            tot += (int64_t)widths[l] * ((widths[l + 1] + 31) & ~31);
        }
        std::vector<float> th(tot, 0.f), tl(tot, 0.f);
        for (int l = 0; l < L; ++l) {
            const int K = widths[l + 1], Nn = widths[l], ldk = (K + 31) & ~31;
            for (int nn = 0; nn < Nn; ++nn)
                for (int kk = 0; kk < K; ++kk) {
                    const float x = hw[N.Woff[l] + (int64_t)kk * Nn + nn];
                    const float h = tf32(x);
                    th[offs[l] + (int64_t)nn * ldk + kk] = h;
                    tl[offs[l] + (int64_t)nn * ldk + kk] = tf32(x - h);
                }
        }
        dev_free(c, (void*&)c->dWTh, 0);
        dev_free(c, (void*&)c->dWTl, 0);
        dev_free(c, (void*&)c->dA2h, 0);
        dev_free(c, (void*&)c->dA2l, 0);
        dev_free(c, (void*&)c->dA2ph, 0);
        dev_free(c, (void*&)c->dA2pl, 0);
        TRY(dev_alloc(c, c->dWTh, tot));
        TRY(dev_alloc(c, c->dWTl, tot));
        std::vector<float> a2h, a2l, a2ph, a2pl;
        if (L >= 2) {
            const int K = widths[1], R2 = widths[2], ldk = (K + 31) & ~31, nk = ldk / 32;
            const size_t m1 = (size_t)((R2 + 127) / 128) * 128, m2 = (size_t)((2 * R2 + 127) / 128) * 128;
            a2h.assign(m1 * ldk, 0.f);
            a2l.assign(m1 * ldk, 0.f);
            a2ph.assign(m2 * ldk, 0.f);
            a2pl.assign(m2 * ldk, 0.f);
            for (int ii = 0; ii < R2; ++ii)
                for (int kk = 0; kk < K; ++kk) {
                    const float x = hw[N.Woff[1] + (int64_t)ii * K + kk];
                    const float xp = x > 0.f ? x : 0.f, xn = x < 0.f ? x : 0.f;
                    const int64_t o = tc::blk_index(ii, kk, nk), op = tc::blk_index(ii, kk, nk),
                                  on = tc::blk_index(R2 + ii, kk, nk);
                    a2h[o] = tf32(x);
                    a2l[o] = tf32(x - a2h[o]);
                    a2ph[op] = tf32(xp);
                    a2pl[op] = tf32(xp - a2ph[op]);
                    a2ph[on] = tf32(xn);
                    a2pl[on] = tf32(xn - a2ph[on]);
                }
            TRY(dev_alloc(c, c->dA2h, a2h.size()));
            TRY(dev_alloc(c, c->dA2l, a2l.size()));
            TRY(dev_alloc(c, c->dA2ph, a2ph.size()));
            TRY(dev_alloc(c, c->dA2pl, a2pl.size()));
            CUDA_TRY(c, cudaMemcpyAsync(c->dA2h, a2h.data(), a2h.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(c->dA2l, a2l.data(), a2l.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(c->dA2ph, a2ph.data(), a2ph.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(c->dA2pl, a2pl.data(), a2pl.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        }
        {
            // reverse-sweep copies: W_l row-major with K = n_{l-1} padded to 32 (TF32 parts), and W_l in
            // the kept-level layout (rows padded to 32)
            int64_t rt = 0, lt = 0;
            for (int l = 0; l < L; ++l) {
                c->WRoff[l] = rt;
                c->WLoff[l] = lt;
                rt += (int64_t)widths[l + 1] * ((widths[l] + 31) & ~31);
                lt += (int64_t)((widths[l + 1] + 127) & ~127) * ((widths[l] + 31) & ~31);
            }
            std::vector<float> rh(rt, 0.f), rl(rt, 0.f), lv(lt, 0.f);
            for (int l = 0; l < L; ++l) {
                const int rows = widths[l + 1], K = widths[l], ldk = (K + 31) & ~31;
                for (int i = 0; i < rows; ++i)
                    for (int k = 0; k < K; ++k) {
                        const float x = hw[N.Woff[l] + (int64_t)i * K + k];
                        const float h = tf32(x);
                        rh[c->WRoff[l] + (int64_t)i * ldk + k] = h;
                        rl[c->WRoff[l] + (int64_t)i * ldk + k] = tf32(x - h);
                        lv[c->WLoff[l] + tc::blk_index(i, k, ldk >> 5)] = x;
                    }
            }
            dev_free(c, (void*&)c->dWRh, 0);
            dev_free(c, (void*&)c->dWRl, 0);
            dev_free(c, (void*&)c->dWlev, 0);
            TRY(dev_alloc(c, c->dWRh, rt));
            TRY(dev_alloc(c, c->dWRl, rt));
            TRY(dev_alloc(c, c->dWlev, lt));
            CUDA_TRY(c, cudaMemcpyAsync(c->dWRh, rh.data(), rt * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(c->dWRl, rl.data(), rt * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(c->dWlev, lv.data(), lt * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        }
        if (!c->derr) TRY(dev_alloc(c, c->derr, 1));
        CUDA_TRY(c, cudaMemcpyAsync(c->dWTh, th.data(), tot * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(c->dWTl, tl.data(), tot * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        for (int l = 0; l < L; ++l) c->WToff[l] = offs[l];
    }
    const int oldH = c->H;
    c->net = N;
    c->net.H = oldH;
    c->has_ctrl = true;
    if (c->dalpha) {
        dev_free(c, (void*&)c->dalpha, 0);
        c->alpha_set = false;
    }
    return DR_OK;
}

int dr_load_dynamics(dr_ctx* c, int n, int m, const double* A, const double* B, const double* e) {
    if (!c || !A || !B) return fail(c, DR_ERR_ARG, "dr_load_dynamics: NULL argument");
    if (n < 1 || m < 1 || n > 64 || m > 64) return fail(c, DR_ERR_SHAPE, "n = %d, m = %d (supported 1..64)", n, m);
    if (c->has_ctrl && (c->net.n != n || c->net.m != m))
        return fail(c, DR_ERR_SHAPE, "dynamics (n=%d, m=%d) do not match controller (n=%d, m=%d)", n, m, c->net.n, c->net.m);
    for (int i = 0; i < n * n; ++i)
        if (!std::isfinite(A[i])) return fail(c, DR_ERR_NONFINITE, "non-finite A");
    for (int i = 0; i < n * m; ++i)
        if (!std::isfinite(B[i])) return fail(c, DR_ERR_NONFINITE, "non-finite B");
    std::vector<double> he(n, 0.0);
    if (e)
        for (int i = 0; i < n; ++i) {
            if (!std::isfinite(e[i])) return fail(c, DR_ERR_NONFINITE, "non-finite e");
            he[i] = e[i];
        }
    CUDA_TRY(c, cudaSetDevice(c->device));
    dev_free(c, (void*&)c->dA, 0);
    dev_free(c, (void*&)c->dB, 0);
    dev_free(c, (void*&)c->de, 0);
    c->gshift_valid = false;  // gradients of the previous dynamics
    c->gtheta_valid = false;
    TRY(dev_alloc(c, c->dA, (size_t)n * n));
    TRY(dev_alloc(c, c->dB, (size_t)n * m));
    TRY(dev_alloc(c, c->de, (size_t)n));
    CUDA_TRY(c, cudaMemcpyAsync(c->dA, A, sizeof(double) * n * n, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->dB, B, sizeof(double) * n * m, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->de, he.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (!c->has_ctrl) {
        c->net.n = n;
        c->net.m = m;
    }
    c->has_dyn = true;
    return DR_OK;
}

static void clear_domain_state(dr_ctx* c) {
    free_outputs(c);
    dev_free(c, (void*&)c->deoff, 0);
    dev_free(c, (void*&)c->dsp_row, 0);
    dev_free(c, (void*&)c->dsp, 0);
    dev_free(c, (void*&)c->dbeta, 0);
    dev_free(c, (void*&)c->dalpha, 0);
    c->nnz = 0;
    c->alpha_set = false;
    if (c->opt.slope_mode == DR_SLOPE_USER) c->opt.slope_mode = DR_SLOPE_CHORD;
}

int dr_set_boxes(dr_ctx* c, int64_t D, const double* lo, const double* hi, int on_device) {
    if (!c) return DR_ERR_ARG;
    if (D < 0) return fail(c, DR_ERR_ARG, "D = %lld", (long long)D);
    if (D > 0 && (!lo || !hi)) return fail(c, DR_ERR_ARG, "dr_set_boxes: NULL lo/hi");
    if (!c->has_ctrl && !c->has_dyn) return fail(c, DR_ERR_STATE, "load the controller or dynamics before the boxes");
    const int n = c->net.n;
    if (!on_device)
        for (int64_t i = 0; i < D * n; ++i) {
            if (!std::isfinite(lo[i]) || !std::isfinite(hi[i])) return fail(c, DR_ERR_NONFINITE, "non-finite box");
            if (lo[i] > hi[i]) return fail(c, DR_ERR_ARG, "box %lld has lo > hi", (long long)(i / n));
        }
    CUDA_TRY(c, cudaSetDevice(c->device));
    if (D > 0 && D == c->D && c->dlo0 && c->dhi0) {
        // same domain count: keep the box and output buffers (and any captured graph); the
        // per-domain splits, slopes and step offsets are reset as for new boxes
        dev_free(c, (void*&)c->deoff, 0);
        dev_free(c, (void*&)c->dsp_row, 0);
        dev_free(c, (void*&)c->dsp, 0);
        dev_free(c, (void*&)c->dbeta, 0);
        dev_free(c, (void*&)c->dalpha, 0);
        c->nnz = 0;
        c->alpha_set = false;
        if (c->opt.slope_mode == DR_SLOPE_USER) c->opt.slope_mode = DR_SLOPE_CHORD;
    } else {
        clear_domain_state(c);
        dev_free(c, (void*&)c->dlo0, 0);
        dev_free(c, (void*&)c->dhi0, 0);
        c->D = D;
        TRY(dev_alloc(c, c->dlo0, (size_t)D * n));
        TRY(dev_alloc(c, c->dhi0, (size_t)D * n));
    }
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (D > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(c->dlo0, lo, sizeof(double) * D * n, k, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(c->dhi0, hi, sizeof(double) * D * n, k, c->stream));
    }
    if (!on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DR_OK;
}

int dr_set_splits(dr_ctx* c, const int64_t* row_ptr, const dr_split* s, const float* beta) {
    if (!c || !row_ptr) return fail(c, DR_ERR_ARG, "dr_set_splits: NULL row_ptr");
    if (!c->has_ctrl) return fail(c, DR_ERR_STATE, "load the controller before the splits");
    const int64_t D = c->D;
    if (row_ptr[0] != 0) return fail(c, DR_ERR_ARG, "row_ptr[0] must be 0");
    for (int64_t d = 0; d < D; ++d)
        if (row_ptr[d + 1] < row_ptr[d]) return fail(c, DR_ERR_ARG, "row_ptr decreases at %lld", (long long)d);
    const int64_t nnz = row_ptr[D];
    if (nnz > 0 && !s) return fail(c, DR_ERR_ARG, "NULL split array with nnz = %lld", (long long)nnz);
    if (nnz > (int64_t)0x7fffffff) return fail(c, DR_ERR_SHAPE, "too many splits");
    const int L = c->net.L;
    for (int64_t d = 0; d < D; ++d) {
        for (int64_t k = row_ptr[d]; k < row_ptr[d + 1]; ++k) {
            const dr_split& r = s[k];
            if (r.layer < 1 || r.layer > L - 1) return fail(c, DR_ERR_ARG, "split %lld: layer %d not hidden", (long long)k, r.layer);
            if (r.neuron < 0 || r.neuron >= c->net.w[r.layer])
                return fail(c, DR_ERR_ARG, "split %lld: neuron %d out of range", (long long)k, r.neuron);
            if (r.t < 0) return fail(c, DR_ERR_ARG, "split %lld: t = %d", (long long)k, r.t);
            if (r.sign != 1 && r.sign != -1) return fail(c, DR_ERR_ARG, "split %lld: sign %d", (long long)k, r.sign);
            if (k > row_ptr[d]) {
                const dr_split& q = s[k - 1];
                if (q.t > r.t || (q.t == r.t && q.layer > r.layer))
                    return fail(c, DR_ERR_ARG, "splits of domain %lld not sorted by (t, layer)", (long long)d);
            }
            if (beta && !(beta[k] >= 0.f && std::isfinite(beta[k])))
                return fail(c, DR_ERR_ARG, "beta[%lld] must be finite and >= 0", (long long)k);
        }
    }
    CUDA_TRY(c, cudaSetDevice(c->device));
    dev_free(c, (void*&)c->dsp_row, 0);
    dev_free(c, (void*&)c->dsp, 0);
    dev_free(c, (void*&)c->dbeta, 0);
    TRY(dev_alloc(c, c->dsp_row, (size_t)D + 1));
    TRY(dev_alloc(c, c->dsp, (size_t)nnz));
    TRY(dev_alloc(c, c->dbeta, (size_t)nnz));
    CUDA_TRY(c, cudaMemcpyAsync(c->dsp_row, row_ptr, sizeof(int64_t) * (D + 1), cudaMemcpyHostToDevice, c->stream));
    if (nnz) {
        static_assert(sizeof(dr_split) == sizeof(SplitRec), "split layout");
        CUDA_TRY(c, cudaMemcpyAsync(c->dsp, s, sizeof(SplitRec) * nnz, cudaMemcpyHostToDevice, c->stream));
        if (beta) CUDA_TRY(c, cudaMemcpyAsync(c->dbeta, beta, sizeof(float) * nnz, cudaMemcpyHostToDevice, c->stream));
        else CUDA_TRY(c, cudaMemsetAsync(c->dbeta, 0, sizeof(float) * nnz, c->stream));
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->nnz = nnz;
    return DR_OK;
}

int dr_set_horizon(dr_ctx* c, int H) {
    if (!c) return DR_ERR_ARG;
    if (H < 1 || H > 100000) return fail(c, DR_ERR_ARG, "H = %d", H);
    if (H != c->H) {
        free_outputs(c);
        dev_free(c, (void*&)c->deoff, 0);
        dev_free(c, (void*&)c->dalpha, 0);
        c->alpha_set = false;
        if (c->opt.slope_mode == DR_SLOPE_USER) c->opt.slope_mode = DR_SLOPE_CHORD;
    }
    c->H = H;
    c->net.H = H;
    return DR_OK;
}

static int check_ready(dr_ctx* c) {
    if (!c->has_ctrl) return fail(c, DR_ERR_STATE, "controller not loaded");
    if (!c->has_dyn) return fail(c, DR_ERR_STATE, "dynamics not loaded");
    if (c->H < 1) return fail(c, DR_ERR_STATE, "horizon not set");
    if (c->net.n != c->net.w[0] || c->net.m != c->net.w[c->net.L]) return fail(c, DR_ERR_SHAPE, "controller/dynamics mismatch");
    return DR_OK;
}

static int ensure_outputs(dr_ctx* c) {
    const int n = c->net.n;
    const size_t ob = sizeof(double) * (size_t)c->D * (c->H + 1) * n;
    if (c->dout_lo && c->out_bytes == ob) return DR_OK;
    free_outputs(c);
    TRY(dev_alloc(c, c->dout_lo, ob / sizeof(double)));
    TRY(dev_alloc(c, c->dout_hi, ob / sizeof(double)));
    c->out_bytes = ob;
    TRY(dev_alloc(c, c->dV, (size_t)c->D));
    TRY(dev_alloc(c, c->dstatus, (size_t)c->D));
    TRY(dev_alloc(c, c->dhull, 2 * (size_t)(c->H + 1) * n));
    return DR_OK;
}

static int tape_stride(const NetDesc& N) { return N.n * N.n + 4 * N.n + 2; }

static int ensure_tape(dr_ctx* c) {
    const size_t tb = sizeof(double) * (size_t)c->D * c->H * tape_stride(c->net);
    if (c->dtape && c->tape_bytes == tb) return DR_OK;
    dev_free(c, (void*&)c->dtape, c->tape_bytes);
    TRY(dev_alloc(c, c->dtape, tb / sizeof(double)));
    c->tape_bytes = tb;
    return DR_OK;
}

// ------------------------------------------------------------------------------------------------
// staged (wide) path
// ------------------------------------------------------------------------------------------------

static int64_t wide_lam_stride(const NetDesc& N) {
    int64_t best = 1;
    for (int l = 2; l <= N.L; ++l)
        for (int k = 0; k <= l - 1; ++k) best = std::max<int64_t>(best, (int64_t)N.w[l] * ((N.w[k] + 31) & ~31));
    return best;
}

// Intercept partial sets per stacked row of a GEMM with NN output columns: (column tiles) x (column
// groups per tile), the largest over the tile widths the GEMM autotuner may pick (128, 64, 32).
static int64_t gemm_part_sets(int NN) {
    int64_t best = 0;
    for (int bn : {tc_bn(NN), 128, 64, 32}) best = std::max<int64_t>(best, (int64_t)((NN + bn - 1) / bn) * tc::epi_groups(bn));
    return best;
}

static int64_t wide_part_per_domain(const NetDesc& N) {
    int64_t best = 1;
    for (int l = 2; l <= N.L; ++l)
        for (int mm = l - 1; mm >= 2; --mm) best = std::max<int64_t>(best, (int64_t)N.w[l] * gemm_part_sets(N.w[mm - 1]));
    return best;
}

// Partial Lambda_x rows per stacked row when the last chain level is fused into the GEMM epilogue
// (one per column tile, for any tile width the autotuner may pick).
static int wide_lx_parts(const NetDesc& N) { return (int)gemm_part_sets(N.w[1]); }

static size_t wide_bytes_per_domain(const NetDesc& N) {
    const int n = N.n, m = N.m;
    size_t b = 0;
    b += sizeof(double) * (n + n * n + n + n + n + 2);           // c, P, Ilo, Ihi, v, w, vacc
    b += sizeof(int) + sizeof(uint32_t);                          // cursor, status
    b += sizeof(float) * (n + n * n + n + n + n + 1);            // FP32 view
    b += sizeof(float) * 4 * std::max(N.hidden, 1);               // l, u, s, d
    b += sizeof(double) * 2 * N.maxw;                             // kappa (FP64)
    b += sizeof(double) * N.maxw + sizeof(float) * (n + std::max(N.hidden, 1));  // rigorous mode: kerr, xmax, q
    b += sizeof(float);                                                           // Taylor-model scale
    b += sizeof(float) * ((size_t)N.maxw * n + 4 * N.maxw);       // G, a, R, S
    b += sizeof(double) * 3 * m;                                  // controller TM (FP64)
    b += sizeof(float) * 4 * wide_lam_stride(N);                  // Lambda buffers (two TF32 pairs)
    b += sizeof(float) * 3 * wide_part_per_domain(N);             // intercept partials of fused levels
    b += sizeof(float) * (size_t)N.maxw * wide_lx_parts(N) * n;   // partial Lambda_x rows of a fused final level
    if (N.L >= 2) {                                                // target-2 GEMM operands and results
        const size_t ldk1 = (N.w[1] + 31) & ~31;
        b += sizeof(float) * (2 * (n + 1) * ldk1 + 2 * ldk1 + (size_t)N.w[2] * (n + 1) + 2 * (size_t)N.w[2]);
    }
    return b + 16 * 24;
}

// Carve the chunk scratch for Dc domains out of one allocation.
// Extra floats per Lambda buffer: the blocked operand layout pads the stacked rows to whole
// 128-row tiles.
static int64_t wide_lam_pad(const NetDesc& N) {
    int ldk = 32;
    for (int l = 0; l <= N.L; ++l) ldk = std::max(ldk, (N.w[l] + 31) & ~31);
    return (int64_t)tc::BM * ldk;
}

struct T2Scratch {
    float *Bh, *Bl, *Dh, *Dl, *C1, *C2;
};

static int wide_bind(dr_ctx* c, WideArgs& a, int Dc, int lanes, int lane, float** lamA, float** lamB, float** lamC,
                     float** lamD, float** part, float** lxpart, T2Scratch* t2) {
    const NetDesc& N = a.net;
    // + 256 B of alignment for each of the (fewer than 64) buffers carved below, whatever Dc is
    const size_t need = (wide_bytes_per_domain(N) * (size_t)Dc + 4 * sizeof(float) * wide_lam_pad(N) + 64 * 256 + 255) & ~size_t(255);
    if (!c->wscratch || c->wscratch_bytes < need * lanes || c->wDc != Dc || c->wLanes != lanes) {
        dev_free(c, c->wscratch, c->wscratch_bytes);
        c->wscratch_bytes = 0;
        unsigned char* p = nullptr;
        TRY(dev_alloc(c, p, need * lanes));
        c->wscratch = p;
        c->wscratch_bytes = need * lanes;
        c->wDc = Dc;
        c->wLanes = lanes;
    }
    unsigned char* base = reinterpret_cast<unsigned char*>(c->wscratch) + need * lane;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~size_t(255);
        void* r = base + off;
        off += bytes;
        return r;
    };
    const int n = N.n, m = N.m;
    const size_t D = (size_t)Dc;
    a.c = (double*)take(sizeof(double) * D * n);
    a.P = (double*)take(sizeof(double) * D * n * n);
    a.Ilo = (double*)take(sizeof(double) * D * n);
    a.Ihi = (double*)take(sizeof(double) * D * n);
    a.v = (double*)take(sizeof(double) * D * n);
    a.w = (double*)take(sizeof(double) * D);
    a.vacc = (double*)take(sizeof(double) * D);
    a.cursor = (int*)take(sizeof(int) * D);
    a.st = (uint32_t*)take(sizeof(uint32_t) * D);
    a.cf = (float*)take(sizeof(float) * D * n);
    a.Pf = (float*)take(sizeof(float) * D * n * n);
    a.Ilof = (float*)take(sizeof(float) * D * n);
    a.Ihif = (float*)take(sizeof(float) * D * n);
    a.vf = (float*)take(sizeof(float) * D * (n + 1));
    const size_t hid = std::max(N.hidden, 1);
    a.hl = (float*)take(sizeof(float) * D * hid);
    a.hu = (float*)take(sizeof(float) * D * hid);
    a.hs = (float*)take(sizeof(float) * D * hid);
    a.hd = (float*)take(sizeof(float) * D * hid);
    a.klo = (double*)take(sizeof(double) * D * N.maxw);
    a.khi = (double*)take(sizeof(double) * D * N.maxw);
    a.G = (float*)take(sizeof(float) * D * N.maxw * n);
    a.sa = (float*)take(sizeof(float) * D * N.maxw);
    a.sRlo = (float*)take(sizeof(float) * D * N.maxw);
    a.sRhi = (float*)take(sizeof(float) * D * N.maxw);
    a.sS = (float*)take(sizeof(float) * D * N.maxw);
    a.cu = (double*)take(sizeof(double) * D * m);
    a.Iulo = (double*)take(sizeof(double) * D * m);
    a.Iuhi = (double*)take(sizeof(double) * D * m);
    a.kerr = (double*)take(sizeof(double) * D * N.maxw);
    a.xmax = (float*)take(sizeof(float) * D * n);
    a.hq = (float*)take(sizeof(float) * D * hid);
    a.xscale = (float*)take(sizeof(float) * D);
    a.lam_stride = wide_lam_stride(N);
    const int64_t lam_pad = wide_lam_pad(N);
    *lamA = (float*)take(sizeof(float) * (D * a.lam_stride + lam_pad));
    *lamB = (float*)take(sizeof(float) * (D * a.lam_stride + lam_pad));
    *lamC = (float*)take(sizeof(float) * (D * a.lam_stride + lam_pad));
    *lamD = (float*)take(sizeof(float) * (D * a.lam_stride + lam_pad));
    *part = (float*)take(sizeof(float) * D * 3 * wide_part_per_domain(N));
    *lxpart = (float*)take(sizeof(float) * D * N.maxw * wide_lx_parts(N) * n);
    memset(t2, 0, sizeof(*t2));
    if (N.L >= 2) {
        const size_t ldk1 = (N.w[1] + 31) & ~31, NB = n + 1;
        t2->Bh = (float*)take(sizeof(float) * D * NB * ldk1);
        t2->Bl = (float*)take(sizeof(float) * D * NB * ldk1);
        t2->Dh = (float*)take(sizeof(float) * D * ldk1);
        t2->Dl = (float*)take(sizeof(float) * D * ldk1);
        t2->C1 = (float*)take(sizeof(float) * (size_t)N.w[2] * D * NB);
        t2->C2 = (float*)take(sizeof(float) * 2 * (size_t)N.w[2] * D);
    }
    if (off > need) return fail(c, DR_ERR_OOM, "staged scratch layout overflow");
    return DR_OK;
}

// Domains per lane chunk: the option if set, else the fewest equal chunks per lane that a scratch
// budget allows.  The budget is 24 GiB (larger chunks mean longer GEMM launches with fewer partial
// waves), at most a quarter of the free device memory and at most the memory cap left, and never
// below 1 GiB.
static int wide_chunk(dr_ctx* c, const NetDesc& N, int lanes) {
    if (c->opt.chunk_domains > 0) return (int)std::min<int64_t>(std::min<int64_t>(c->opt.chunk_domains, c->D), 65535);
    // a captured pass repeats the plain pass before it: keep its chunk, and query no device state
    // while the stream is being captured
    if (c->capturing && c->wDc > 0 && c->wLanes == lanes) return c->wDc;
    size_t total = size_t(24) << 30;
    size_t free_b = 0, all_b = 0;
    // the scratch this context already holds counts as free, so the choice is stable across calls
    if (cudaMemGetInfo(&free_b, &all_b) == cudaSuccess) total = std::min(total, (free_b + c->wscratch_bytes) / 4);
    if (c->opt.mem_cap_bytes > 0)
        total = std::min(total, (size_t)c->opt.mem_cap_bytes > c->owned ? (size_t)c->opt.mem_cap_bytes - c->owned : size_t(0));
    total = std::max(total, size_t(1) << 30);
    const size_t budget = total / lanes;
    const int64_t dmax = std::min<int64_t>(std::max<int64_t>(1, (int64_t)(budget / wide_bytes_per_domain(N))), 65535);
    // as few chunks per lane as the budget allows, all of (nearly) the same size: a small last chunk
    // would run its GEMMs with few tiles per SM
    const int64_t per_lane = (c->D + lanes - 1) / lanes;
    const int64_t k = (per_lane + dmax - 1) / dmax;
    return (int)std::max<int64_t>(1, (per_lane + k - 1) / k);
}

static inline unsigned blocks_for(int64_t threads, int bs) { return (unsigned)((threads + bs - 1) / bs); }

// Concretisation launch: one thread per row for large row counts (whole-line loads of the
// entry-major Lambda_x partials), four per row for small ones (a shorter dependent chain per row).
static void launch_t_project(dr_ctx* c, const WideArgs& a, int ell, const float* Lx, int shared_lx, int64_t R, int lx_parts,
                             cudaStream_t st, const float* part = nullptr, int ntiles = 0) {
    if (a.net.n <= 16 && R < (int64_t)148 * 128) {
        const unsigned blocks = (unsigned)((R + 63) / 64);
        if (a.net.n % 4 == 0) k_t_project4<true><<<blocks, 256, 0, st>>>(a, ell, Lx, shared_lx, lx_parts, part, ntiles);
        else k_t_project4<false><<<blocks, 256, 0, st>>>(a, ell, Lx, shared_lx, lx_parts, part, ntiles);
    } else {
        // one row per thread (no grid-stride tail); seven blocks of 128 threads per SM at 72 registers
        // (k_t_project's launch bounds): 1.3x the earlier 96-register, 16-blocks-per-SM grid
        const unsigned blocks = (unsigned)std::min<int64_t>((R + 127) / 128, (int64_t)1 << 30);
        if (a.net.n <= 16) k_t_project<16><<<blocks, 128, 0, st>>>(a, ell, Lx, shared_lx, lx_parts, part, ntiles);
        else k_t_project<64><<<blocks, 128, 0, st>>>(a, ell, Lx, shared_lx, lx_parts, part, ntiles);
    }
    c->launches++;
}

// The tensor-core pipeline's error flag (a bounded wait that expired) after the work on the stream.
static int check_tc_error(dr_ctx* c) {
    int herr = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&herr, c->derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (herr) return fail(c, DR_ERR_TIMEOUT, "a tensor-core pipeline wait timed out");
    return DR_OK;
}

// One lane of the staged path: a chunk of domains with its own scratch, advanced on its own stream.
struct WideLane {
    WideArgs a;
    float *lamA, *lamB, *lamC, *lamD, *part, *lxpart;
    T2Scratch t2;
    cudaStream_t st;
    bool active;
};

// Keep mode of the staged forward pass: where one step's chain levels go.  Level Lambda^(m) of target
// ell (m = 1 .. ell-2, the levels a chain GEMM produces) sits at base + off[ell][m], blocked like the
// GEMM operands (tc::blk_index over the chunk's stacked rows, ru32(n_m) columns).
struct KeepLevels {
    float* base;
    int64_t off[DR_MAXL + 1][DR_MAXL + 1];
};

// Every kernel of time step t of one lane's chunk (layers, chain, concretisation, relaxation, dynamics).
// With kl set (keep mode; w.a's keep fields set by the caller) the step also keeps what the staged
// reverse sweep reads.
static int wide_step(dr_ctx* c, WideLane& w, int t, bool tcore, const KeepLevels* kl = nullptr) {
    const NetDesc& N = w.a.net;
    const int n = N.n, L = N.L;
    WideArgs& a = w.a;
    const cudaStream_t st = w.st;
    const int dc = a.Dc;
    float *lamA = w.lamA, *lamB = w.lamB, *lamC = w.lamC, *lamD = w.lamD, *part = w.part, *lxpart = w.lxpart;
    const size_t dyn_smem = sizeof(double) * (n * n + 3 * n + 128);
    k_w_view<<<dc, 128, 0, st>>>(a);
    c->launches++;
    if (a.rigorous && L >= 2) {  // q_1 = |W_1| xmax for the error bounds of the last chain level
        k_r_q<<<blocks_for((int64_t)dc * N.w[1] * 32, 256), 256, 0, st>>>(a, 1);
        c->launches++;
    }
    auto levp = [&](int ell, int mm) -> float* { return kl ? kl->base + kl->off[ell][mm] : nullptr; };
    for (int ell = 1; ell <= L; ++ell) {
        const int rows = N.w[ell];
        const int64_t warps = (int64_t)dc * rows;
        WideArgs ap = a;  // the projection's copy: keep-mode row offset of this target
        ap.koff = ell < L ? N.hoff[ell] : N.hidden;
        if (tcore && ell == 1) {
            // layer 1: Lambda_x = W_1, shared by every domain
            launch_t_project(c, ap, 1, c->dW + N.Woff[0], 1, (int64_t)dc * rows, 0, st);
        } else if (!tcore || ell == 1) {
            k_w_chain_init<<<blocks_for(warps * 32, 256), 256, 0, st>>>(a, ell, lamA);
            c->launches++;
            float* cur = lamA;
            float* nxt = lamB;
            for (int mm = ell - 1; mm >= 1; --mm) {
                const int K = N.w[mm], NN = N.w[mm - 1];
                const float* Wm = c->dW + N.Woff[mm - 1];
                dim3 grid((NN + 63) / 64, (rows + 63) / 64, dc);
                k_w_gemm_simt<<<grid, 256, 0, st>>>(cur, Wm, nxt, rows, K, NN, a.lam_stride);
                c->launches++;
                if (mm - 1 >= 1) {
                    k_w_level_epi<<<blocks_for(warps * 32, 256), 256, 0, st>>>(a, ell, mm - 1, nxt, levp(ell, mm - 1));
                    c->launches++;
                }
                std::swap(cur, nxt);
            }
            if (ell == 1) k_w_project<<<blocks_for(warps * 32, 256), 256, 0, st>>>(ap, 1, c->dW + N.Woff[0], 1);
            else k_w_project<<<blocks_for(warps * 32, 256), 256, 0, st>>>(ap, ell, cur, 0);
            c->launches++;
        } else {
            // tensor-core chain: rows of all domains stacked, A as TF32 parts, shared W^T parts;
            // levels that feed another level form the next operand in the GEMM epilogue, and
            // the last level (x W_1, n columns) is folded into the epilogue of the level before
            const int R = dc * rows;
            const bool fuse_final = N.n <= tc::kFinalCols && tc_bn(N.w[1]) >= 32;
            if (ell == 2) {
                // target 2: two GEMMs with the shared W_2 (and its sign parts) as the left operand
                const int ldk1 = round_up32(N.w[1]), NB = N.n + 1;
                k_t2_prep<<<blocks_for((int64_t)dc * ldk1, 256), 256, 0, st>>>(a, ldk1, w.t2.Bh, w.t2.Bl, w.t2.Dh, w.t2.Dl);
                c->launches++;
                TRY(tc_gemm(c, c->dA2h, c->dA2l, w.t2.Bh, w.t2.Bl, w.t2.C1, rows, N.w[1], dc * NB, ldk1, dc * NB, c->derr, st));
                TRY(tc_gemm(c, c->dA2ph, c->dA2pl, w.t2.Dh, w.t2.Dl, w.t2.C2, 2 * rows, N.w[1], dc, ldk1, dc, c->derr, st));
                if (NB <= kT2MaxNB) {
                    const dim3 grid((unsigned)((dc + kT2TileDoms - 1) / kT2TileDoms), (unsigned)((rows + kT2TileRows - 1) / kT2TileRows));
                    k_t2_finish_tiled<<<grid, 256, 0, st>>>(a, w.t2.C1, w.t2.C2, lamC);
                } else {
                    k_t2_finish<<<blocks_for((int64_t)R, 256), 256, 0, st>>>(a, w.t2.C1, w.t2.C2, lamC);
                }
                c->launches++;
                launch_t_project(c, ap, ell, lamC, 0, R, 0, st);
            } else {
                int ldk = round_up32(N.w[ell - 1]);
                const int K0 = N.w[ell - 1];
                // the register-cached form for K = 128 or 256 without padding, with 16-byte aligned W
                // rows, per-domain vectors and bias (the buffers' bases are 256-byte aligned).  Measured
                // on 1,048,576 rows of K = 256: 380 us against 590 us for the row-per-warp kernel (whose
                // per-row index arithmetic and vector loads bound it); with K = 512 the row-per-warp
                // kernel is already bound by its HBM writes and the register-cached one, at 100
                // registers and two blocks per SM, took 1040 us against 554.
                const bool rc = K0 == ldk && (K0 == 128 || K0 == 256) && N.Woff[ell - 1] % 4 == 0 && N.hidden % 4 == 0 &&
                                N.hoff[ell - 1] % 4 == 0 && N.boff[ell - 2] % 4 == 0;
                const unsigned rcb = (unsigned)((warps + kChainInitThreads / 32 * kChainRowsPerWarp - 1) /
                                                (kChainInitThreads / 32 * kChainRowsPerWarp));
                if (rc && K0 == 128) k_t_chain_init_rc<1><<<rcb, kChainInitThreads, 0, st>>>(a, ell, lamA, lamB, ldk);
                else if (rc) k_t_chain_init_rc<2><<<rcb, kChainInitThreads, 0, st>>>(a, ell, lamA, lamB, ldk);
                else k_t_chain_init<<<blocks_for(warps * 32, kChainInitThreads), kChainInitThreads, 0, st>>>(a, ell, lamA, lamB, ldk);
                c->launches++;
                float *curh = lamA, *curl = lamB, *nxth = lamC, *nxtl = lamD;
                int lx_parts = 0, fin_tiles = 0;
                for (int mm = ell - 1; mm >= 1; --mm) {
                    const int K = N.w[mm], NN = N.w[mm - 1];
                    const float* WTh = c->dWTh + c->WToff[mm - 1];
                    const float* WTl = c->dWTl + c->WToff[mm - 1];
                    if (mm - 1 >= 1) {
                        const bool fin = mm == 2 && fuse_final;
                        tc::ChainEpi epi{};
                        epi.hs = a.hs;
                        epi.hd = a.hd;
                        epi.bias = c->db + N.boff[mm - 2];
                        epi.hidden = N.hidden;
                        epi.hoff = N.hoff[mm - 1];
                        epi.rows_per_dom = rows;
                        epi.Ah = nxth;
                        epi.Al = nxtl;
                        epi.ldk = round_up32(NN);
                        epi.part = part;
                        epi.lev = levp(ell, mm - 1);
                        if (fin) {
                            epi.W1 = c->dW + N.Woff[0];
                            epi.n0 = N.n;
                            epi.lxpart = lxpart;
                        }
                        int bn = 0;
                        TRY(tc_gemm(c, curh, curl, WTh, WTl, nullptr, R, K, NN, ldk, 0, c->derr, st, &epi, &bn));
                        const int gx = (NN + bn - 1) / bn;  // column tiles of the GEMM as launched
                        const int ntiles = gx * tc::epi_groups(bn);
                        if (fin) {
                            lx_parts = gx;        // one Lambda_x partial per column tile
                            fin_tiles = ntiles;   // its intercept partials are added by the projection
                            break;
                        }
                        k_t_partials<<<blocks_for(R, 256), 256, 0, st>>>(a, ell, part, ntiles);
                        c->launches++;
                        std::swap(curh, nxth);
                        std::swap(curl, nxtl);
                        ldk = round_up32(NN);
                    } else {
                        TRY(tc_gemm(c, curh, curl, WTh, WTl, nxth, R, K, NN, ldk, NN, c->derr, st));
                    }
                }
                launch_t_project(c, ap, ell, lx_parts ? lxpart : nxth, 0, R, lx_parts, st, part, fin_tiles);
            }
        }
        if (ell < L) {
            k_w_relax<<<dc, 256, 0, st>>>(a, ell, t);
            c->launches++;
            if (a.rigorous && ell + 1 <= L - 1) {
                k_r_q<<<blocks_for((int64_t)dc * N.w[ell + 1] * 32, 256), 256, 0, st>>>(a, ell + 1);
                c->launches++;
            }
        }
    }
    k_w_dyn<<<dc, 128, dyn_smem, st>>>(a, t);
    c->launches++;
    CUDA_TRY(c, cudaGetLastError());
    return DR_OK;
}

static int run_forward_wide(dr_ctx* c, int mode, float* alpha_used) {
    NetDesc N = c->net;
    N.H = c->H;
    const int n = N.n, H = N.H;
    WideArgs a;
    memset(&a, 0, sizeof(a));
    a.net = N;
    a.W = c->dW;
    a.b = c->db;
    a.A = c->dA;
    a.B = c->dB;
    a.e = c->de;
    a.eoff = c->deoff;
    a.lo0 = c->dlo0;
    a.hi0 = c->dhi0;
    a.sp_row = c->nnz ? c->dsp_row : nullptr;
    a.sp = c->dsp;
    a.beta = c->dbeta;
    a.alpha = c->dalpha;
    a.mode = mode;
    a.rho = (float)c->opt.margin_rho;
    a.box_margin = c->opt.box_margin;
    a.lo = c->dout_lo;
    a.hi = c->dout_hi;
    a.V = c->dV;
    a.status = c->dstatus;
    a.alpha_used = alpha_used;
    a.rigorous = c->opt.rigorous;
    // Domains are independent: two lanes of chunks advance on two streams, so that one lane's
    // memory-bound kernels overlap the other lane's tensor-core GEMMs.
    const int lanes = c->D >= 256 ? 2 : 1;
    const int Dc = (int)std::min<int64_t>(wide_chunk(c, N, lanes), (c->D + lanes - 1) / lanes);
    WideLane w[dr_ctx::kMaxLanes];
    for (int l = 0; l < lanes; ++l) {
        w[l].a = a;
        TRY(wide_bind(c, w[l].a, Dc, lanes, l, &w[l].lamA, &w[l].lamB, &w[l].lamC, &w[l].lamD, &w[l].part, &w[l].lxpart,
                      &w[l].t2));
        w[l].st = c->stream;
    }
    // rigorous mode runs the chain on CUDA cores: its error bounds use the IEEE FP32 round-to-nearest
    // model, which the tensor cores' internal accumulation does not document
    const bool tcore = c->opt.precision != DR_PREC_SIMT && !c->opt.rigorous;
    if (tcore) CUDA_TRY(c, cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream));
    if (lanes > 1) {
        if (!c->ev_fork) CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
        CUDA_TRY(c, cudaEventRecord(c->ev_fork, c->stream));
        for (int l = 1; l < lanes; ++l) {
            if (!c->aux[l]) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->aux[l], cudaStreamNonBlocking));
            if (!c->ev_join[l]) CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_join[l], cudaEventDisableTiming));
            CUDA_TRY(c, cudaStreamWaitEvent(c->aux[l], c->ev_fork, 0));
            w[l].st = c->aux[l];
        }
    }
    int rc = DR_OK;
    for (int64_t d0 = 0; d0 < c->D && rc == DR_OK; d0 += (int64_t)lanes * Dc) {
        for (int l = 0; l < lanes; ++l) {
            const int64_t s0 = d0 + (int64_t)l * Dc;
            w[l].active = s0 < c->D;
            if (!w[l].active) continue;
            w[l].a.d0 = s0;
            w[l].a.Dc = (int)std::min<int64_t>(Dc, c->D - s0);
            k_w_seed<<<blocks_for((int64_t)w[l].a.Dc * n, 256), 256, 0, w[l].st>>>(w[l].a);
            c->launches++;
        }
        for (int t = 0; t < H && rc == DR_OK; ++t)
            for (int l = 0; l < lanes && rc == DR_OK; ++l)
                if (w[l].active) rc = wide_step(c, w[l], t, tcore);
    }
    for (int l = 1; l < lanes; ++l) {
        // join the other lanes back into the context's stream (also on the error path)
        cudaEventRecord(c->ev_join[l], c->aux[l]);
        cudaStreamWaitEvent(c->stream, c->ev_join[l], 0);
    }
    if (rc != DR_OK) return rc;
    c->last_tc = tcore;
    if (tcore && !c->capturing) TRY(check_tc_error(c));  // a captured pass is checked after each replay
    return DR_OK;
}

// The shared padded weights of slab mode (same offsets as the shared-memory layout's weight region).
static int ensure_wpad(dr_ctx* c, const NetDesc& N, const FusedLayout& Y) {
    if (c->dWpad) return DR_OK;
    TRY(dev_alloc(c, c->dWpad, (size_t)(Y.bs - Y.Ws[0]) / sizeof(float)));
    k_pad_weights<<<296, 256, 0, c->stream>>>(N, Y, c->dW, c->dWpad);
    CUDA_TRY(c, cudaGetLastError());
    c->launches++;
    return DR_OK;
}

// Domains per launch and the slab buffer for running the fused kernels out of global memory.
// Slab budget: 8 GiB (enough for two CTAs per SM of the widest controllers), at most a quarter of the
// free device memory (the context's own slabs counted as free), never below 1 GiB.
static int slab_chunk(dr_ctx* c, size_t per_cta, int64_t* chunk) {
    if (c->capturing && c->gslab && c->gslab_bytes >= per_cta) {
        // inside a graph capture: reuse the slab of the plain run before it (no device query, no allocation)
        *chunk = std::min<int64_t>(std::min<int64_t>(c->D, (int64_t)(c->gslab_bytes / std::max<size_t>(per_cta, 1))), 4 * 148);
        return DR_OK;
    }
    size_t budget = size_t(8) << 30;
    size_t free_b = 0, all_b = 0;
    if (cudaMemGetInfo(&free_b, &all_b) == cudaSuccess) budget = std::min(budget, (free_b + c->gslab_bytes) / 4);
    budget = std::max(budget, size_t(1) << 30);
    int64_t ch = std::max<int64_t>(1, std::min<int64_t>(c->D, (int64_t)(budget / std::max<size_t>(per_cta, 1))));
    ch = std::min<int64_t>(ch, 4 * 148);
    const size_t need = (size_t)ch * per_cta;
    if (!c->gslab || c->gslab_bytes < need) {
        dev_free(c, (void*&)c->gslab, c->gslab_bytes);
        c->gslab_bytes = 0;
        TRY(dev_alloc(c, c->gslab, need));
        c->gslab_bytes = need;
    }
    *chunk = ch;
    return DR_OK;
}

// Forward pass over all domains into the library-owned buffers (optionally recording the tape
// and the slopes in effect).  Bounds-only passes: the fused kernels serve controllers that fit in
// shared memory (DR_PREC_AUTO); DR_PREC_SIMT / DR_PREC_TF32X3 and wider controllers take the
// staged path.
static bool use_fused(const dr_ctx* c) {
    return c->opt.precision == DR_PREC_AUTO && !c->opt.rigorous && fused_fits(c->net);
}

static int run_forward(dr_ctx* c, int mode, float* alpha_used, bool tape) {
    NetDesc N = c->net;
    N.H = c->H;
    if (c->D == 0) return DR_OK;
    if (mode == DR_SLOPE_USER && !c->dalpha) return fail(c, DR_ERR_STATE, "no slopes set");
    // The tape-recording pass always runs the fused kernel; a controller whose working set exceeds
    // shared memory runs it out of per-CTA global slabs.
    if (!tape && !use_fused(c)) return run_forward_wide(c, mode, alpha_used);
    const bool slab = fused_layout(N).total > kMaxSmem;
    if (!tape && multi_layout(N, 1).total <= kMaxSmem) {
        // grouped kernel: G domains per CTA, (threads, G) chosen by the autotuner
        MultiArgs a;
        memset(&a, 0, sizeof(a));
        a.net = N;
        a.W = c->dW;
        a.b = c->db;
        a.A = c->dA;
        a.B = c->dB;
        a.e = c->de;
        a.eoff = c->deoff;
        a.lo0 = c->dlo0;
        a.hi0 = c->dhi0;
        a.D = c->D;
        a.sp_row = c->nnz ? c->dsp_row : nullptr;
        a.sp = c->dsp;
        a.beta = c->dbeta;
        a.alpha = c->dalpha;
        a.mode = mode;
        a.rho = (float)c->opt.margin_rho;
        a.box_margin = c->opt.box_margin;
        a.lo = c->dout_lo;
        a.hi = c->dout_hi;
        a.V = c->dV;
        a.status = c->dstatus;
        a.alpha_used = alpha_used;
        int variant = 0;
        TRY(tuned_variant(c, a, &variant));
        TRY(launch_multi(c, a, variant));
        return DR_OK;
    }
    if (tape) TRY(ensure_tape(c));
    FusedArgs a;
    memset(&a, 0, sizeof(a));
    a.net = N;
    a.lay = fused_layout(N);
    a.W = c->dW;
    a.b = c->db;
    a.A = c->dA;
    a.B = c->dB;
    a.e = c->de;
    a.eoff = c->deoff;
    a.lo0 = c->dlo0;
    a.hi0 = c->dhi0;
    a.sp_row = c->nnz ? c->dsp_row : nullptr;
    a.sp = c->dsp;
    a.beta = c->dbeta;
    a.alpha = c->dalpha;
    a.mode = mode;
    a.rho = (float)c->opt.margin_rho;
    a.box_margin = c->opt.box_margin;
    a.lo = c->dout_lo;
    a.hi = c->dout_hi;
    a.V = c->dV;
    a.status = c->dstatus;
    a.alpha_used = alpha_used;
    a.tape = tape ? c->dtape : nullptr;
    a.tape_stride = tape_stride(N);
    const int nt = fused_threads(N);
    int smem = a.lay.total;
    int64_t chunk = 1 << 20;
    if (slab) {
        a.slab_stride = ((int64_t)a.lay.total + 255) & ~int64_t(255);
        TRY(slab_chunk(c, (size_t)a.slab_stride, &chunk));
        TRY(ensure_wpad(c, N, a.lay));
        a.gslab = c->gslab;
        a.gwpad = c->dWpad;
        smem = nt == 256 ? (int)(sizeof(float) * kSlabTileFloats) : 0;  // the chain products' tiles
    }
    for (int64_t d0 = 0; d0 < c->D; d0 += chunk) {
        a.d0 = d0;
        const int64_t nd = std::min(chunk, c->D - d0);
        if (nt == 128) {
            CUDA_TRY(c, cudaFuncSetAttribute(k_fused_forward<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            k_fused_forward<128><<<(unsigned)nd, 128, smem, c->stream>>>(a);
        } else {
            CUDA_TRY(c, cudaFuncSetAttribute(k_fused_forward<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            k_fused_forward<256><<<(unsigned)nd, 256, smem, c->stream>>>(a);
        }
        CUDA_TRY(c, cudaGetLastError());
        c->launches++;
    }
    return DR_OK;
}

int dr_compute_bounds(dr_ctx* c, double* lo, double* hi, double* hull_lo, double* hull_hi, uint32_t* status,
                      int out_on_device) {
    if (!c) return DR_ERR_ARG;
    TRY(check_ready(c));
    CUDA_TRY(c, cudaSetDevice(c->device));
    TRY(ensure_outputs(c));
    if (c->opt.slope_mode == DR_SLOPE_USER && !c->alpha_set) return fail(c, DR_ERR_STATE, "DR_SLOPE_USER without slopes");
    const int n = c->net.n, H = c->H;
    const int TN = (H + 1) * n;
    const int mode = c->opt.slope_mode, hull = (hull_lo || hull_hi) ? 1 : 0;
    auto pass = [&]() -> int {
        TRY(run_forward(c, mode, nullptr, false));
        if (c->D > 0 && hull) {
            k_hull<<<TN, 256, 0, c->stream>>>(c->dout_lo, c->dout_hi, c->dstatus, c->D, TN, c->dhull, c->dhull + TN);
            CUDA_TRY(c, cudaGetLastError());
            c->launches++;
        }
        return DR_OK;
    };
    const bool graphs = c->opt.graphs == 0 && !c->opt.timing && !c->graphs_broken && c->stream != nullptr && c->D > 0;
    if (graphs && c->gexec && c->g_epoch == c->epoch && c->g_mode == mode && c->g_hull == hull) {
        CUDA_TRY(c, cudaGraphLaunch(c->gexec, c->stream));
        c->launches += c->graph_launches;
        c->graph_replays++;
        if (c->g_check_tc) TRY(check_tc_error(c));
    } else if (graphs && c->seen_epoch == c->epoch && c->seen_mode == mode && c->seen_hull == hull) {
        // second call with unchanged state: capture the pass (its first run already tuned and allocated)
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        const int64_t l0 = c->launches;
        int rc = DR_OK;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            c->capturing = true;
            rc = pass();
            c->capturing = false;
            const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
            if (rc == DR_OK && e == cudaSuccess && g && cudaGraphInstantiate(&c->gexec, g, 0) == cudaSuccess) {
                c->g_epoch = c->epoch;
                c->g_mode = mode;
                c->g_hull = hull;
                c->g_check_tc = c->last_tc;
                c->graph_launches = c->launches - l0;
            } else {
                c->gexec = nullptr;
            }
            if (g) cudaGraphDestroy(g);
        }
        if (!c->gexec) {
            // capture is not possible here: plain launches from now on
            cudaGetLastError();
            c->graphs_broken = true;
            c->launches = l0;
            TRY(pass());
        } else {
            CUDA_TRY(c, cudaGraphLaunch(c->gexec, c->stream));
            if (c->g_check_tc) TRY(check_tc_error(c));
        }
    } else {
        TRY(pass());
        c->seen_epoch = c->epoch;
        c->seen_mode = mode;
        c->seen_hull = hull;
    }
    const size_t ob = sizeof(double) * (size_t)c->D * TN;
    const cudaMemcpyKind k = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (c->D > 0) {
        if (lo) CUDA_TRY(c, cudaMemcpyAsync(lo, c->dout_lo, ob, k, c->stream));
        if (hi) CUDA_TRY(c, cudaMemcpyAsync(hi, c->dout_hi, ob, k, c->stream));
        if (status) CUDA_TRY(c, cudaMemcpyAsync(status, c->dstatus, sizeof(uint32_t) * c->D, k, c->stream));
        if (hull_lo) CUDA_TRY(c, cudaMemcpyAsync(hull_lo, c->dhull, sizeof(double) * TN, k, c->stream));
        if (hull_hi) CUDA_TRY(c, cudaMemcpyAsync(hull_hi, c->dhull + TN, sizeof(double) * TN, k, c->stream));
    }
    if (!out_on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DR_OK;
}

int dr_get_objective(dr_ctx* c, double* V, int on_device) {
    if (!c || !V) return fail(c, DR_ERR_ARG, "dr_get_objective: NULL");
    if (!c->dV) return fail(c, DR_ERR_STATE, "no bounds computed yet");
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaMemcpyAsync(V, c->dV, sizeof(double) * c->D, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
    if (!on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DR_OK;
}

static int ensure_alpha(dr_ctx* c) {
    if (c->dalpha) return DR_OK;
    return dev_alloc(c, c->dalpha, (size_t)c->D * c->H * std::max(c->net.hidden, 1));
}

int dr_get_alpha(dr_ctx* c, float* alpha, int on_device) {
    if (!c || !alpha) return fail(c, DR_ERR_ARG, "dr_get_alpha: NULL");
    TRY(check_ready(c));
    CUDA_TRY(c, cudaSetDevice(c->device));
    const size_t cnt = (size_t)c->D * c->H * c->net.hidden;
    if (!c->alpha_set) {
        // the slopes in effect for the current mode
        TRY(ensure_outputs(c));
        TRY(ensure_alpha(c));
        TRY(run_forward(c, c->opt.slope_mode, c->dalpha, false));
    }
    CUDA_TRY(c, cudaMemcpyAsync(alpha, c->dalpha, sizeof(float) * cnt, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DR_OK;
}

int dr_set_alpha(dr_ctx* c, const float* alpha, int on_device) {
    if (!c || !alpha) return fail(c, DR_ERR_ARG, "dr_set_alpha: NULL");
    TRY(check_ready(c));
    CUDA_TRY(c, cudaSetDevice(c->device));
    TRY(ensure_alpha(c));
    const size_t cnt = (size_t)c->D * c->H * c->net.hidden;
    if (!on_device)
        for (size_t i = 0; i < cnt; ++i)
            if (!(alpha[i] >= 0.f && alpha[i] <= 1.f)) return fail(c, DR_ERR_ARG, "alpha[%zu] = %g outside [0, 1]", i, alpha[i]);
    CUDA_TRY(c, cudaMemcpyAsync(c->dalpha, alpha, sizeof(float) * cnt, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->alpha_set = true;
    c->opt.slope_mode = DR_SLOPE_USER;
    return DR_OK;
}

int dr_get_beta(dr_ctx* c, float* beta, int on_device) {
    if (!c || (!beta && c->nnz)) return fail(c, DR_ERR_ARG, "dr_get_beta: NULL");
    if (!c->nnz) return DR_OK;
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaMemcpyAsync(beta, c->dbeta, sizeof(float) * c->nnz, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DR_OK;
}

int dr_set_beta(dr_ctx* c, const float* beta, int on_device) {
    if (!c || (!beta && c->nnz)) return fail(c, DR_ERR_ARG, "dr_set_beta: NULL");
    if (!c->nnz) return DR_OK;
    if (!on_device)
        for (int64_t k = 0; k < c->nnz; ++k)
            if (!(beta[k] >= 0.f && std::isfinite(beta[k]))) return fail(c, DR_ERR_ARG, "beta[%lld] must be finite and >= 0", (long long)k);
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaMemcpyAsync(c->dbeta, beta, sizeof(float) * c->nnz, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DR_OK;
}

// Controller parameter counts: packed weights (layer after layer, row-major) and packed biases.
static int64_t theta_weights(const NetDesc& N) {
    return N.Woff[N.L - 1] + (int64_t)N.w[N.L] * N.w[N.L - 1];
}
static int64_t theta_biases(const NetDesc& N) {
    return N.boff[N.L - 1] + N.w[N.L];
}
constexpr int kThetaGroups = 64;                        // partial sums of the slice reduction
constexpr size_t kThetaSliceBytes = size_t(512) << 20;  // per-domain slices of one backward chunk

static int launch_backward(dr_ctx* c, int mode, const double* wlo, const double* whi, float* galpha, float* gbeta,
                           double* gshift = nullptr, bool wgrad = false) {
    NetDesc N = c->net;
    N.H = c->H;
    if (c->D == 0) return DR_OK;
    FusedArgs a;
    memset(&a, 0, sizeof(a));
    a.net = N;
    a.lay = fused_layout(N, true, wgrad);
    const bool slab = a.lay.total > kMaxSmem;
    a.W = c->dW;
    a.b = c->db;
    a.A = c->dA;
    a.B = c->dB;
    a.e = c->de;
    a.eoff = c->deoff;
    a.lo0 = c->dlo0;
    a.hi0 = c->dhi0;
    a.sp_row = c->nnz ? c->dsp_row : nullptr;
    a.sp = c->dsp;
    a.beta = c->dbeta;
    a.alpha = c->dalpha;
    a.mode = mode;
    a.rho = (float)c->opt.margin_rho;
    a.tape = c->dtape;
    a.tape_stride = tape_stride(N);
    a.wlo = wlo;
    a.whi = whi;
    a.dalpha = galpha;
    a.dbeta = gbeta;
    a.gshift = gshift;
    const int nt = fused_threads(N);
    int smem = a.lay.total;
    int64_t chunk = 1 << 20;
    if (slab) {
        a.slab_stride = ((int64_t)a.lay.total + 255) & ~int64_t(255);
        TRY(slab_chunk(c, (size_t)a.slab_stride, &chunk));
        TRY(ensure_wpad(c, N, a.lay));
        a.gslab = c->gslab;
        a.gwpad = c->dWpad;
        smem = nt == 256 ? (int)(sizeof(float) * kSlabTileFloats) : 0;  // the chain products' tiles
    }
    if (c->opt.chunk_domains > 0) chunk = std::min<int64_t>(chunk, c->opt.chunk_domains);
    const int64_t nth = theta_weights(N) + theta_biases(N);
    if (wgrad) {
        // one slice of dV/dtheta per domain (the kernel runs a CTA per domain), summed after each chunk
        a.gth_boff = theta_weights(N);
        a.gth_stride = (nth + 63) & ~int64_t(63);
        chunk = std::max<int64_t>(1, std::min<int64_t>(chunk, (int64_t)(kThetaSliceBytes / (sizeof(float) * a.gth_stride))));
        const size_t need = sizeof(float) * (size_t)std::min(chunk, c->D) * a.gth_stride;
        if (c->gth_bytes < need) {
            dev_free(c, (void*&)c->dgth, c->gth_bytes);
            c->gth_bytes = 0;
            TRY(dev_alloc(c, c->dgth, need / sizeof(float)));
            c->gth_bytes = need;
        }
        dev_free(c, (void*&)c->dgth_part, 0);
        TRY(dev_alloc(c, c->dgth_part, (size_t)kThetaGroups * nth));
        if (!c->dgtheta) TRY(dev_alloc(c, c->dgtheta, (size_t)nth));
        CUDA_TRY(c, cudaMemsetAsync(c->dgtheta, 0, sizeof(double) * nth, c->stream));
    }
    for (int64_t d0 = 0; d0 < c->D; d0 += chunk) {
        a.d0 = d0;
        const int64_t nd = std::min(chunk, c->D - d0);
        if (wgrad) {
            a.gth = c->dgth;
            CUDA_TRY(c, cudaMemsetAsync(c->dgth, 0, sizeof(float) * nd * a.gth_stride, c->stream));
        }
        if (nt == 128) {
            CUDA_TRY(c, cudaFuncSetAttribute(k_fused_backward<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            k_fused_backward<128><<<(unsigned)nd, 128, smem, c->stream>>>(a);
        } else {
            CUDA_TRY(c, cudaFuncSetAttribute(k_fused_backward<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            k_fused_backward<256><<<(unsigned)nd, 256, smem, c->stream>>>(a);
        }
        CUDA_TRY(c, cudaGetLastError());
        c->launches++;
        if (wgrad) {
            const int groups = (int)std::min<int64_t>(kThetaGroups, nd);
            const unsigned gx = (unsigned)((nth + 255) / 256);
            k_theta_partial<<<dim3(gx, (unsigned)groups), 256, 0, c->stream>>>(c->dgth, nd, a.gth_stride, nth, c->dgth_part);
            k_theta_finish<<<gx, 256, 0, c->stream>>>(c->dgth_part, groups, nth, c->dgtheta);
            CUDA_TRY(c, cudaGetLastError());
            c->launches += 2;
        }
    }
    return DR_OK;
}

// ------------------------------------------------------------------------------------------------
// staged reverse sweep (wide controllers): keep-mode forward pass of a chunk, then the reverse
// ------------------------------------------------------------------------------------------------

// The keep store (one slot per step) and the adjoint scratch of one chunk of Dc domains, carved from
// one allocation.  With base == nullptr only the size is computed.
struct RevStore {
    // keep slots: array x at x + t * sx
    float *Pf, *cf, *Ilof, *Ihif, *vsnap, *hl, *hu, *hs, *hd, *hl0, *hu0, *Gk, *LXk, *lev;
    int64_t sPf, sn, svs, shid, sG, slev;
    KeepLevels kl;  // level offsets inside a slot (base unset)
    double* tape;   // [Dc][H+1][ts]
    // adjoint state
    double *gcn, *gPn, *gIlon, *gIhin, *gv, *gw;  // carried across steps (contiguous, zeroed per chunk)
    size_t carried_bytes;
    double *gc, *gP, *gIlo, *gIhi, *gcu, *gPu, *gIulo, *gIuhi;
    float *gs, *gd, *ga, *gklo, *gkhi, *gRlo, *gRhi, *gG, *gLx, *gLxh, *gLxl, *gLa, *gLb, *colpart;
    float *Lh[2], *Ll[2];
    int ldw;
};

// Shared memory limit of the few-rows CUDA-core chain reverse (k_rv_chain_rows).
constexpr size_t kRevRowsSmem = 96 * 1024;

// Targets whose chain reverse runs on the tensor cores: the reverse epilogue sums columns over row
// segments inside one domain, 32 rows each or a whole domain of 2, 4, 8 or 16 rows.
static bool rev_tc_rows(int rows) { return rows % 32 == 0 || (rows >= 2 && rows < 32 && (rows & (rows - 1)) == 0); }

// Row count of the widest target whose chain reverse runs on CUDA cores (0 if none).
static int rev_simt_rows(const NetDesc& N, bool tc_rev) {
    int r = 0;
    for (int ell = 2; ell <= N.L; ++ell)
        if (!tc_rev || !rev_tc_rows(N.w[ell])) r = std::max(r, N.w[ell]);
    return r;
}

static size_t rev_store(const NetDesc& N, int Dc, bool tc_rev, RevStore* S, unsigned char* base) {
    const int n = N.n, m = N.m, L = N.L, H = N.H;
    const int64_t D = Dc, hid = std::max(N.hidden, 1), krows = N.hidden + m;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        off = (off + 255) & ~size_t(255);
        void* r = base ? base + off : nullptr;
        off += bytes;
        return r;
    };
    S->sPf = D * n * n;
    S->sn = D * n;
    S->svs = D * L * (n + 1);
    S->shid = D * hid;
    S->sG = D * krows * n;
    int64_t lt = 0;
    for (int ell = 0; ell <= DR_MAXL; ++ell)
        for (int mm = 0; mm <= DR_MAXL; ++mm) S->kl.off[ell][mm] = 0;
    for (int ell = 3; ell <= L; ++ell)
        for (int mm = 1; mm <= ell - 2; ++mm) {
            S->kl.off[ell][mm] = lt;
            lt += (((D * N.w[ell]) + tc::BM - 1) / tc::BM * tc::BM) * ((N.w[mm] + 31) & ~31);
        }
    S->slev = std::max<int64_t>(lt, 1);
    S->kl.base = nullptr;
    const size_t f = sizeof(float);
    S->Pf = (float*)take(f * H * S->sPf);
    S->cf = (float*)take(f * H * S->sn);
    S->Ilof = (float*)take(f * H * S->sn);
    S->Ihif = (float*)take(f * H * S->sn);
    S->vsnap = (float*)take(f * H * S->svs);
    S->hl = (float*)take(f * H * S->shid);
    S->hu = (float*)take(f * H * S->shid);
    S->hs = (float*)take(f * H * S->shid);
    S->hd = (float*)take(f * H * S->shid);
    S->hl0 = (float*)take(f * H * S->shid);
    S->hu0 = (float*)take(f * H * S->shid);
    S->Gk = (float*)take(f * H * S->sG);
    S->LXk = (float*)take(f * H * S->sG);
    S->lev = (float*)take(f * H * S->slev);
    const int ts = tape_stride(N);
    S->tape = (double*)take(sizeof(double) * D * (H + 1) * ts);
    // carried adjoints: one contiguous block
    off = (off + 255) & ~size_t(255);
    const size_t c0 = off;
    double* cb = (double*)(base ? base + off : nullptr);
    off += sizeof(double) * D * (4 * n + n * n + n + 1);
    S->carried_bytes = off - c0;
    S->gcn = cb;
    S->gPn = cb ? cb + D * n : nullptr;
    S->gIlon = cb ? S->gPn + D * n * n : nullptr;
    S->gIhin = cb ? S->gIlon + D * n : nullptr;
    S->gv = cb ? S->gIhin + D * n : nullptr;
    S->gw = cb ? S->gv + D * n : nullptr;
    const size_t dd = sizeof(double);
    S->gc = (double*)take(dd * D * n);
    S->gP = (double*)take(dd * D * n * n);
    S->gIlo = (double*)take(dd * D * n);
    S->gIhi = (double*)take(dd * D * n);
    S->gcu = (double*)take(dd * D * m);
    S->gPu = (double*)take(dd * D * m * n);
    S->gIulo = (double*)take(dd * D * m);
    S->gIuhi = (double*)take(dd * D * m);
    S->gs = (float*)take(f * D * hid);
    S->gd = (float*)take(f * D * hid);
    S->ga = (float*)take(f * D * N.maxw);
    S->gklo = (float*)take(f * D * N.maxw);
    S->gkhi = (float*)take(f * D * N.maxw);
    S->gRlo = (float*)take(f * D * N.maxw);
    S->gRhi = (float*)take(f * D * N.maxw);
    S->gG = (float*)take(f * D * N.maxw * n);
    S->gLx = (float*)take(f * D * N.maxw * n);
    const int64_t rpad = ((D * N.maxw + tc::BM - 1) / tc::BM) * tc::BM;
    const int ldkx = (n + 31) & ~31;
    int ldkw = 32;
    for (int l = 1; l < L; ++l) ldkw = std::max(ldkw, (N.w[l] + 31) & ~31);
    S->gLxh = (float*)take(f * rpad * ldkx);
    S->gLxl = (float*)take(f * rpad * ldkx);
    for (int q = 0; q < 2; ++q) {
        S->Lh[q] = (float*)take(f * rpad * ldkw);
        S->Ll[q] = (float*)take(f * rpad * ldkw);
    }
    S->colpart = (float*)take(f * D * std::max(1, (N.maxw + 31) / 32) * 2 * N.maxw);  // [segments][2][n_m]
    S->ldw = std::max(N.maxw, n);
    const int sr = rev_simt_rows(N, tc_rev);
    S->gLa = (float*)take(f * D * std::max(sr, 1) * S->ldw);
    S->gLb = (float*)take(f * D * std::max(sr, 1) * S->ldw);
    return off + 256;
}

// Domains per chunk of the staged reverse sweep: the keep store, the adjoint scratch and the forward
// scratch of a chunk within min(96 GiB, half the free memory, the memory cap left), at least one.
static int rev_chunk(dr_ctx* c, const NetDesc& N, bool tc_rev) {
    if (c->opt.chunk_domains > 0) return (int)std::min<int64_t>(std::min<int64_t>(c->opt.chunk_domains, c->D), 65535);
    if (c->capturing && c->wDc > 0) return c->wDc;  // a captured step repeats the plain step before it
    RevStore S;
    const size_t per = rev_store(N, 64, tc_rev, &S, nullptr) / 64 + wide_bytes_per_domain(N) + 4096;
    size_t budget = size_t(96) << 30;
    size_t free_b = 0, all_b = 0;
    if (cudaMemGetInfo(&free_b, &all_b) == cudaSuccess) budget = std::min(budget, (free_b + c->kscratch_bytes + c->wscratch_bytes) / 2);
    if (c->opt.mem_cap_bytes > 0)
        budget = std::min(budget, (size_t)c->opt.mem_cap_bytes > c->owned ? (size_t)c->opt.mem_cap_bytes - c->owned : size_t(0));
    const int64_t dmax = std::min<int64_t>(std::max<int64_t>(1, (int64_t)(budget / per)), 65535);
    const int64_t k = (c->D + dmax - 1) / dmax;  // equal chunks
    return (int)std::max<int64_t>(1, (c->D + k - 1) / k);
}

static bool use_staged_reverse(const dr_ctx* c, bool wgrad) {
    NetDesc N = c->net;
    N.H = c->H;
    if (wgrad || c->opt.reverse == 1) return false;
    return c->opt.reverse == 2 || fused_layout(N, true, false).total > kMaxSmem;
}

// Forward pass with the slopes of `mode` (outputs lo/hi/V/status as dr_compute_bounds writes them)
// and the reverse sweep, chunk by chunk, for controllers too wide for the fused kernels.
static int run_staged_backward(dr_ctx* c, int mode, const double* wlo, const double* whi, float* galpha, float* gbeta,
                               double* gshift) {
    NetDesc N = c->net;
    N.H = c->H;
    const int n = N.n, L = N.L, H = N.H;
    if (c->D == 0) return DR_OK;
    if (mode == DR_SLOPE_USER && !c->dalpha) return fail(c, DR_ERR_STATE, "no slopes set");
    const bool tcore = c->opt.precision != DR_PREC_SIMT;
    const bool tc_rev = tcore && persistent_gemm_usable<3>();
    const int Dc = rev_chunk(c, N, tc_rev);
    WideArgs a;
    memset(&a, 0, sizeof(a));
    a.net = N;
    a.W = c->dW;
    a.b = c->db;
    a.A = c->dA;
    a.B = c->dB;
    a.e = c->de;
    a.eoff = c->deoff;
    a.lo0 = c->dlo0;
    a.hi0 = c->dhi0;
    a.sp_row = c->nnz ? c->dsp_row : nullptr;
    a.sp = c->dsp;
    a.beta = c->dbeta;
    a.alpha = c->dalpha;
    a.mode = mode;
    a.rho = (float)c->opt.margin_rho;
    a.box_margin = c->opt.box_margin;
    a.lo = c->dout_lo;
    a.hi = c->dout_hi;
    a.V = c->dV;
    a.status = c->dstatus;
    WideLane w;
    w.a = a;
    TRY(wide_bind(c, w.a, Dc, 1, 0, &w.lamA, &w.lamB, &w.lamC, &w.lamD, &w.part, &w.lxpart, &w.t2));
    w.st = c->stream;
    RevStore S;
    const size_t need = rev_store(N, Dc, tc_rev, &S, nullptr);
    if (!c->kscratch || c->kscratch_bytes < need) {
        dev_free(c, c->kscratch, c->kscratch_bytes);
        c->kscratch_bytes = 0;
        unsigned char* p = nullptr;
        TRY(dev_alloc(c, p, need));
        c->kscratch = p;
        c->kscratch_bytes = need;
    }
    rev_store(N, Dc, tc_rev, &S, reinterpret_cast<unsigned char*>(c->kscratch));
    if (c->nnz && (!c->dsph || c->sph_n != c->nnz)) {
        dev_free(c, (void*&)c->dsph, 0);
        TRY(dev_alloc(c, c->dsph, (size_t)c->nnz));
        c->sph_n = c->nnz;
    }
    const cudaStream_t st = c->stream;
    if (tcore) CUDA_TRY(c, cudaMemsetAsync(c->derr, 0, sizeof(int), st));
    {
        // the first reverse GEMM's left operand: its K padding columns (n .. 31) stay zero
        const size_t gx = sizeof(float) * (size_t)(((int64_t)Dc * N.maxw + tc::BM - 1) / tc::BM * tc::BM) * round_up32(n);
        CUDA_TRY(c, cudaMemsetAsync(S.gLxh, 0, gx, st));
        CUDA_TRY(c, cudaMemsetAsync(S.gLxl, 0, gx, st));
    }
    const int krows = N.hidden + N.m;
    RevArgs r;
    memset(&r, 0, sizeof(r));
    r.net = N;
    r.W = c->dW;
    r.b = c->db;
    r.A = c->dA;
    r.B = c->dB;
    r.sp_row = a.sp_row;
    r.sp = c->dsp;
    r.beta = c->dbeta;
    r.sph = c->dsph;
    r.alpha = c->dalpha;
    r.mode = mode;
    r.wlo = wlo;
    r.whi = whi;
    r.dalpha = galpha;
    r.dbeta = gbeta;
    r.gshift = gshift;
    r.tape = S.tape;
    r.krows = krows;
    r.gcn = S.gcn;
    r.gPn = S.gPn;
    r.gIlon = S.gIlon;
    r.gIhin = S.gIhin;
    r.gv = S.gv;
    r.gw = S.gw;
    r.gc = S.gc;
    r.gP = S.gP;
    r.gIlo = S.gIlo;
    r.gIhi = S.gIhi;
    r.gcu = S.gcu;
    r.gPu = S.gPu;
    r.gIulo = S.gIulo;
    r.gIuhi = S.gIuhi;
    r.gs = S.gs;
    r.gd = S.gd;
    r.ga = S.ga;
    r.gklo = S.gklo;
    r.gkhi = S.gkhi;
    r.gRlo = S.gRlo;
    r.gRhi = S.gRhi;
    r.gG = S.gG;
    r.gLa = S.gLa;
    r.gLb = S.gLb;
    r.ldw = S.ldw;
    for (int64_t d0 = 0; d0 < c->D; d0 += Dc) {
        const int nd = (int)std::min<int64_t>(Dc, c->D - d0);
        w.a.d0 = d0;
        w.a.Dc = nd;
        k_w_seed<<<blocks_for((int64_t)nd * n, 256), 256, 0, st>>>(w.a);
        c->launches++;
        // ---- forward pass of the chunk, keeping every step
        for (int t = 0; t < H; ++t) {
            WideLane ws = w;
            WideArgs& k = ws.a;
            k.Pf = S.Pf + t * S.sPf;
            k.cf = S.cf + t * S.sn;
            k.Ilof = S.Ilof + t * S.sn;
            k.Ihif = S.Ihif + t * S.sn;
            k.hl = S.hl + t * S.shid;
            k.hu = S.hu + t * S.shid;
            k.hs = S.hs + t * S.shid;
            k.hd = S.hd + t * S.shid;
            k.hl0 = S.hl0 + t * S.shid;
            k.hu0 = S.hu0 + t * S.shid;
            k.vsnap = S.vsnap + t * S.svs;
            k.Gk = S.Gk + t * S.sG;
            k.LXk = S.LXk + t * S.sG;
            k.krows = krows;
            k.sph = c->dsph;
            k.tape = S.tape;
            KeepLevels kl = S.kl;
            kl.base = S.lev + t * S.slev;
            k_w_tape<<<nd, 128, 0, st>>>(k, t);
            c->launches++;
            TRY(wide_step(c, ws, t, tcore, &kl));
        }
        {
            WideArgs k = w.a;
            k.tape = S.tape;
            k_w_tape<<<nd, 128, 0, st>>>(k, H);
            c->launches++;
        }
        // ---- reverse sweep
        CUDA_TRY(c, cudaMemsetAsync(S.gcn, 0, S.carried_bytes, st));
        r.d0 = d0;
        r.Dc = nd;
        for (int t = H - 1; t >= 0; --t) {
            r.Pf = S.Pf + t * S.sPf;
            r.cf = S.cf + t * S.sn;
            r.Ilof = S.Ilof + t * S.sn;
            r.Ihif = S.Ihif + t * S.sn;
            r.hl = S.hl + t * S.shid;
            r.hu = S.hu + t * S.shid;
            r.hs = S.hs + t * S.shid;
            r.hd = S.hd + t * S.shid;
            r.hl0 = S.hl0 + t * S.shid;
            r.hu0 = S.hu0 + t * S.shid;
            r.vsnap = S.vsnap + t * S.svs;
            r.Gk = S.Gk + t * S.sG;
            r.LXk = S.LXk + t * S.sG;
            float* levt = S.lev + t * S.slev;
            k_rv_dyn<<<nd, 128, 0, st>>>(r, t);
            c->launches++;
            for (int ell = L; ell >= 1; --ell) {
                const int rows = N.w[ell];
                const bool use_tc = tc_rev && ell >= 2 && rev_tc_rows(rows);
                RevArgs rt = r;
                rt.gLx = use_tc ? nullptr : S.gLx;
                rt.gLxh = use_tc ? S.gLxh : nullptr;
                rt.gLxl = use_tc ? S.gLxl : nullptr;
                const size_t tsm = sizeof(float) * (size_t)rv_target_smem_floats(rows, n);
                if (rv_items_per_thread(n) <= 2) {
                    if (tsm > 48 * 1024) CUDA_TRY(c, cudaFuncSetAttribute(k_rv_target<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
                    k_rv_target<2><<<nd, 256, tsm, st>>>(rt, ell, t);
                } else {
                    if (tsm > 48 * 1024) CUDA_TRY(c, cudaFuncSetAttribute(k_rv_target<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
                    k_rv_target<18><<<nd, 256, tsm, st>>>(rt, ell, t);
                }
                c->launches++;
                if (ell < 2) continue;
                if (use_tc) {
                    const int R = nd * rows;
                    const float* Ah = S.gLxh;
                    const float* Al = S.gLxl;
                    int ldkA = round_up32(n);
                    for (int mm = 1; mm <= ell - 1; ++mm) {
                        const int Kc = N.w[mm - 1], Nc = N.w[mm];
                        const bool top = mm == ell - 1;
                        tc::ChainEpi e{};
                        e.hs = r.hs;
                        e.hd = r.hd;
                        e.bias = c->db + N.boff[mm - 1];
                        e.hidden = N.hidden;
                        e.hoff = N.hoff[mm];
                        e.rows_per_dom = rows;
                        e.Ah = top ? nullptr : S.Lh[mm & 1];
                        e.Al = top ? nullptr : S.Ll[mm & 1];
                        e.ldk = round_up32(Nc);
                        e.rklo = S.gklo;
                        e.rkhi = S.gkhi;
                        e.kld = N.maxw;
                        e.rlev = top ? c->dWlev + c->WLoff[ell - 1] : levt + S.kl.off[ell][mm];
                        e.rlev_shared = top ? 1 : 0;
                        e.colpart = S.colpart;
                        TRY(tc_gemm(c, Ah, Al, c->dWRh + c->WRoff[mm - 1], c->dWRl + c->WRoff[mm - 1], nullptr, R, Kc, Nc, ldkA,
                                    0, c->derr, st, &e));
                        k_rv_colsum<<<blocks_for((int64_t)nd * Nc, 256), 256, 0, st>>>(r, ell, mm, S.colpart);
                        c->launches++;
                        Ah = e.Ah;
                        Al = e.Al;
                        ldkA = e.ldk;
                    }
                } else {
                    RevArgs rc = rt;
                    for (int mm = 0; mm <= DR_MAXL; ++mm) rc.tlev[mm] = nullptr;
                    for (int mm = 1; mm <= ell - 2; ++mm) rc.tlev[mm] = levt + S.kl.off[ell][mm];
                    const size_t rsmem = sizeof(float) * 2 * (size_t)rows * S.ldw;
                    if (rows <= 32 && rsmem <= kRevRowsSmem) {
                        if (rsmem > 48 * 1024)
                            CUDA_TRY(c, cudaFuncSetAttribute(k_rv_chain_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem));
                        k_rv_chain_rows<<<nd, 256, rsmem, st>>>(rc, ell);
                    } else {
                        k_rv_chain_simt<<<nd, 256, 0, st>>>(rc, ell);
                    }
                    c->launches++;
                }
            }
            k_rv_carry<<<blocks_for((int64_t)nd * n, 256), 256, 0, st>>>(r, t);
            c->launches++;
        }
    }
    CUDA_TRY(c, cudaGetLastError());
    if (tcore && !c->capturing) TRY(check_tc_error(c));
    return DR_OK;
}

static int ensure_grad_buffers(dr_ctx* c) {
    const size_t na = (size_t)c->D * c->H * std::max(c->net.hidden, 1);
    if (!c->dgalpha) TRY(dev_alloc(c, c->dgalpha, na));
    if (!c->dgbeta) TRY(dev_alloc(c, c->dgbeta, (size_t)std::max<int64_t>(c->nnz, 1)));
    return DR_OK;
}

int dr_backward(dr_ctx* c, const double* dV_dlo, const double* dV_dhi, float* dalpha, float* dbeta, int on_device) {
    if (!c) return DR_ERR_ARG;
    TRY(check_ready(c));
    CUDA_TRY(c, cudaSetDevice(c->device));
    TRY(ensure_outputs(c));
    TRY(ensure_grad_buffers(c));
    const int mode = c->alpha_set ? DR_SLOPE_USER : c->opt.slope_mode;
    const size_t nw = (size_t)c->D * (c->H + 1) * c->net.n;
    const double* wlo = nullptr;
    const double* whi = nullptr;
    if (dV_dlo || dV_dhi) {
        if (!c->dwlo) TRY(dev_alloc(c, c->dwlo, nw));
        if (!c->dwhi) TRY(dev_alloc(c, c->dwhi, nw));
        const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (dV_dlo) CUDA_TRY(c, cudaMemcpyAsync(c->dwlo, dV_dlo, sizeof(double) * nw, k, c->stream));
        else CUDA_TRY(c, cudaMemsetAsync(c->dwlo, 0, sizeof(double) * nw, c->stream));
        if (dV_dhi) CUDA_TRY(c, cudaMemcpyAsync(c->dwhi, dV_dhi, sizeof(double) * nw, k, c->stream));
        else CUDA_TRY(c, cudaMemsetAsync(c->dwhi, 0, sizeof(double) * nw, c->stream));
        wlo = c->dwlo;
        whi = c->dwhi;
    }
    if (!c->dgshift) TRY(dev_alloc(c, c->dgshift, nw));
    c->gshift_valid = false;
    c->gtheta_valid = false;
    if (use_staged_reverse(c, c->opt.weight_grad != 0)) {
        TRY(run_staged_backward(c, mode, wlo, whi, c->dgalpha, c->dgbeta, c->dgshift));
    } else {
        TRY(run_forward(c, mode, nullptr, true));
        TRY(launch_backward(c, mode, wlo, whi, c->dgalpha, c->dgbeta, c->dgshift, c->opt.weight_grad != 0));
    }
    c->gshift_valid = true;
    c->gtheta_valid = c->opt.weight_grad != 0;
    const size_t na = (size_t)c->D * c->H * c->net.hidden;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (dalpha && na) CUDA_TRY(c, cudaMemcpyAsync(dalpha, c->dgalpha, sizeof(float) * na, k, c->stream));
    if (dbeta && c->nnz) CUDA_TRY(c, cudaMemcpyAsync(dbeta, c->dgbeta, sizeof(float) * c->nnz, k, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DR_OK;
}

int dr_set_step_offsets(dr_ctx* c, const double* eoff, int on_device) {
    if (!c) return DR_ERR_ARG;
    TRY(check_ready(c));
    CUDA_TRY(c, cudaSetDevice(c->device));
    if (!eoff) {
        dev_free(c, (void*&)c->deoff, 0);
        return DR_OK;
    }
    const size_t cnt = (size_t)c->D * c->H * c->net.n;
    if (!on_device)
        for (size_t i = 0; i < cnt; ++i)
            if (!std::isfinite(eoff[i])) return fail(c, DR_ERR_NONFINITE, "non-finite step offset at %zu", i);
    if (c->D == 0) return DR_OK;
    if (!c->deoff) TRY(dev_alloc(c, c->deoff, cnt));
    CUDA_TRY(c, cudaMemcpyAsync(c->deoff, eoff, sizeof(double) * cnt, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                c->stream));
    if (!on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DR_OK;
}

int dr_get_shift_gradient(dr_ctx* c, double* g, int on_device) {
    if (!c || !g) return fail(c, DR_ERR_ARG, "dr_get_shift_gradient: NULL");
    if (!c->gshift_valid || !c->dgshift) return fail(c, DR_ERR_STATE, "no dr_backward since the problem changed");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const size_t cnt = (size_t)c->D * (c->H + 1) * c->net.n;
    CUDA_TRY(c, cudaMemcpyAsync(g, c->dgshift, sizeof(double) * cnt, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
    if (!on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DR_OK;
}

int dr_get_weight_gradient(dr_ctx* c, double* dW, double* db, int on_device) {
    if (!c || (!dW && !db)) return fail(c, DR_ERR_ARG, "dr_get_weight_gradient: NULL");
    if (!c->gtheta_valid || !c->dgtheta)
        return fail(c, DR_ERR_STATE, "no dr_backward with dr_options.weight_grad = 1 since the problem changed");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const int64_t nW = theta_weights(c->net), nb = theta_biases(c->net);
    if (dW) CUDA_TRY(c, cudaMemcpyAsync(dW, c->dgtheta, sizeof(double) * nW, k, c->stream));
    if (db) CUDA_TRY(c, cudaMemcpyAsync(db, c->dgtheta + nW, sizeof(double) * nb, k, c->stream));
    if (!on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DR_OK;
}

int dr_optimize_slopes(dr_ctx* c, int steps, double lr_alpha, double lr_beta, double* V_out) {
    if (!c) return DR_ERR_ARG;
    if (steps < 0 || !(lr_alpha >= 0.0) || !(lr_beta >= 0.0)) return fail(c, DR_ERR_ARG, "steps/learning rates out of range");
    TRY(check_ready(c));
    CUDA_TRY(c, cudaSetDevice(c->device));
    TRY(ensure_outputs(c));
    TRY(ensure_grad_buffers(c));
    if (c->D == 0) return DR_OK;
    const int64_t per_dom = (int64_t)c->H * c->net.hidden;
    const size_t na = (size_t)c->D * per_dom;
    if (!c->alpha_set) {
        TRY(ensure_alpha(c));
        TRY(run_forward(c, DR_SLOPE_CHORD, c->dalpha, false));  // start at the chord slopes
        c->alpha_set = true;
    }
    if (!c->dbest_alpha) TRY(dev_alloc(c, c->dbest_alpha, std::max<size_t>(na, 1)));
    if (!c->dbest_beta) TRY(dev_alloc(c, c->dbest_beta, (size_t)std::max<int64_t>(c->nnz, 1)));
    if (!c->dbestV) TRY(dev_alloc(c, c->dbestV, (size_t)c->D));
    dev_free(c, (void*&)c->dVhist, 0);
    TRY(dev_alloc(c, c->dVhist, (size_t)steps + 1));
    {
        std::vector<double> inf(c->D, std::numeric_limits<double>::infinity());
        CUDA_TRY(c, cudaMemcpyAsync(c->dbestV, inf.data(), sizeof(double) * c->D, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    if (!c->dhist_slot) TRY(dev_alloc(c, c->dhist_slot, 1));
    CUDA_TRY(c, cudaMemsetAsync(c->dhist_slot, 0, sizeof(int), c->stream));
    const int64_t* sp_row = c->nnz ? c->dsp_row : nullptr;
    // evaluation at the current slopes (forward pass, with the tape when a gradient follows), keep-best
    // per domain, and the next V history entry
    auto evaluate = [&](bool tape) -> int {
        TRY(run_forward(c, DR_SLOPE_USER, nullptr, tape));
        k_keep_best<<<(unsigned)c->D, 128, 0, c->stream>>>(c->dV, c->dbestV, c->dalpha, c->dbest_alpha, c->dbeta,
                                                          c->dbest_beta, sp_row, per_dom);
        k_sum_hist<<<1, 256, 0, c->stream>>>(c->dbestV, c->D, c->dVhist, c->dhist_slot);
        CUDA_TRY(c, cudaGetLastError());
        c->launches += 2;
        return DR_OK;
    };
    // one projected-gradient step: evaluate with the tape, reverse sweep, projected updates (the staged
    // reverse sweep runs its own forward pass, whose objective the keep-best step then reads)
    const bool staged = use_staged_reverse(c, false);
    auto step = [&]() -> int {
        if (staged) {
            TRY(run_staged_backward(c, DR_SLOPE_USER, nullptr, nullptr, c->dgalpha, c->dgbeta, nullptr));
            k_keep_best<<<(unsigned)c->D, 128, 0, c->stream>>>(c->dV, c->dbestV, c->dalpha, c->dbest_alpha, c->dbeta,
                                                              c->dbest_beta, sp_row, per_dom);
            k_sum_hist<<<1, 256, 0, c->stream>>>(c->dbestV, c->D, c->dVhist, c->dhist_slot);
            CUDA_TRY(c, cudaGetLastError());
            c->launches += 2;
        } else {
            TRY(evaluate(true));
            TRY(launch_backward(c, DR_SLOPE_USER, nullptr, nullptr, c->dgalpha, c->dgbeta));
        }
        if (na) {
            k_pgd<<<1184, 256, 0, c->stream>>>(c->dalpha, c->dgalpha, (int64_t)na, (float)lr_alpha, 0.f, 1.f);
            c->launches++;
        }
        if (c->nnz && lr_beta > 0.0) {
            k_pgd<<<1184, 256, 0, c->stream>>>(c->dbeta, c->dgbeta, c->nnz, (float)lr_beta, 0.f, INFINITY);
            c->launches++;
        }
        CUDA_TRY(c, cudaGetLastError());
        return DR_OK;
    };
    int it = 0;
    if (steps > 0) {
        TRY(step());  // the first step runs plain: it allocates the tape, slabs and padded weights
        it = 1;
    }
    // The remaining steps issue the same launches on the same buffers: capture one step in a CUDA
    // graph and replay it (needs a stream other than the legacy default stream; if the capture
    // fails, the steps run as plain launches).
    if (steps - it >= 1 && c->opt.graphs == 0 && !c->opt.timing && !c->graphs_broken && c->stream != nullptr) {
        const int64_t l0 = c->launches;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t gx = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            c->capturing = true;
            const int rc = step();
            c->capturing = false;
            const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
            if (rc != DR_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&gx, g, 0) != cudaSuccess) gx = nullptr;
            if (g) cudaGraphDestroy(g);
        }
        const int64_t per_step = c->launches - l0;
        c->launches = l0;
        if (!gx) {
            cudaGetLastError();
        } else {
            int rc = DR_OK;
            for (; it < steps && rc == DR_OK; ++it) {
                const cudaError_t e = cudaGraphLaunch(gx, c->stream);
                if (e != cudaSuccess) rc = fail(c, DR_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
                c->launches += per_step;
                c->graph_replays++;
            }
            cudaGraphExecDestroy(gx);
            if (rc != DR_OK) return rc;
        }
    }
    for (; it < steps; ++it) TRY(step());
    TRY(evaluate(false));
    // install the best slopes and multipliers and leave their bounds in the output buffers
    if (na) CUDA_TRY(c, cudaMemcpyAsync(c->dalpha, c->dbest_alpha, sizeof(float) * na, cudaMemcpyDeviceToDevice, c->stream));
    if (c->nnz) CUDA_TRY(c, cudaMemcpyAsync(c->dbeta, c->dbest_beta, sizeof(float) * c->nnz, cudaMemcpyDeviceToDevice, c->stream));
    c->opt.slope_mode = DR_SLOPE_USER;
    TRY(run_forward(c, DR_SLOPE_USER, nullptr, false));
    if (V_out) CUDA_TRY(c, cudaMemcpyAsync(V_out, c->dVhist, sizeof(double) * (steps + 1), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return DR_OK;
}

}  // extern "C"

// Utility entry: FP32-accurate C = A B^T on tensor cores (temporary device buffers).
extern "C" int dr_tf32x3_gemm(int M, int N, int K, const float* A, const float* BT, float* C, void* stream) {
    if (M < 0 || N < 0 || K < 1 || !A || !BT || !C) return fail(nullptr, DR_ERR_ARG, "dr_tf32x3_gemm: bad arguments");
    if (M == 0 || N == 0) return DR_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int ldk = round_up32(K);
    const int64_t Mpad = ((int64_t)M + tc::BM - 1) / tc::BM * tc::BM;  // blocked A: whole 128-row tiles
    float *Ah = nullptr, *Al = nullptr, *Bh = nullptr, *Bl = nullptr;
    int* err = nullptr;
    auto cleanup = [&]() {
        cudaFree(Ah);
        cudaFree(Al);
        cudaFree(Bh);
        cudaFree(Bl);
        cudaFree(err);
    };
    if (cudaMalloc(&Ah, sizeof(float) * (size_t)Mpad * ldk) != cudaSuccess || cudaMalloc(&Al, sizeof(float) * (size_t)Mpad * ldk) != cudaSuccess ||
        cudaMalloc(&Bh, sizeof(float) * (size_t)N * ldk) != cudaSuccess || cudaMalloc(&Bl, sizeof(float) * (size_t)N * ldk) != cudaSuccess ||
        cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(nullptr, DR_ERR_OOM, "dr_tf32x3_gemm: allocation failed");
    }
    cudaMemsetAsync(err, 0, sizeof(int), st);
    tc::k_split_tf32<<<1184, 256, 0, st>>>(A, K, M, K, ldk, Ah, Al, 1);
    tc::k_split_tf32<<<1184, 256, 0, st>>>(BT, K, N, K, ldk, Bh, Bl, 0);
    int rc = tc_gemm(nullptr, Ah, Al, Bh, Bl, C, M, K, N, ldk, N, err, st);
    int herr = 0;
    if (rc == DR_OK) {
        cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(nullptr, DR_ERR_CUDA, "dr_tf32x3_gemm: %s", cudaGetErrorString(e));
        else if (herr) rc = fail(nullptr, DR_ERR_TIMEOUT, "dr_tf32x3_gemm: a pipeline wait timed out");
    }
    cleanup();
    return rc;
}

// One thread waits on the first phase of a fresh mbarrier that nothing arrives on: the bounded wait
// every pipeline stage uses must give up after its budget and raise the error flag.
__global__ void k_wait_expiry(int* err, long long budget) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!tc::mbar_wait_for(&bar, 0, budget)) atomicExch(err, 1);
    }
}

extern "C" int dr_check_wait_expiry(double seconds) {
    if (!(seconds > 0.0) || seconds > 2.0) return fail(nullptr, DR_ERR_ARG, "dr_check_wait_expiry: seconds must be in (0, 2]");
    int dev = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) {
        cudaGetLastError();
        return fail(nullptr, DR_ERR_CUDA, "dr_check_wait_expiry: no device");
    }
    int* err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, DR_ERR_OOM, "dr_check_wait_expiry: allocation failed");
    }
    int rc = DR_OK, herr = 0;
    cudaMemset(err, 0, sizeof(int));
    k_wait_expiry<<<1, 32>>>(err, (long long)(seconds * 1e3 * khz));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = fail(nullptr, DR_ERR_CUDA, "dr_check_wait_expiry: %s", cudaGetErrorString(e));
    else if (herr) rc = fail(nullptr, DR_ERR_TIMEOUT, "dr_check_wait_expiry: the wait gave up as designed");
    cudaFree(err);
    return rc;
}

// ------------------------------------------------------------------------------------------------
// Allocation-free slope gradient (dr_slope_gradient_static): the reverse sweep with its tape in a
// statically reserved device array instead of context-owned memory.
// ------------------------------------------------------------------------------------------------

#include <mutex>

static __device__ __align__(256) double g_static_tape[DR_STATIC_SCRATCH_BYTES / sizeof(double)];

static std::mutex g_static_mu;
static double* g_static_tape_ptr[64];  // device address of g_static_tape, per device ordinal
static bool g_static_ready[64];

// Host code cannot use g_static_tape directly (it names a host-side shadow); it needs the device
// address, looked up with the device current.  Outside stream capture the address is looked up
// on every call (the module may have been loaded again, e.g. after cudaDeviceReset, at another
// address); inside a capture, where the lookup could load the module and break the capture, the
// address from the last call outside capture on this device is used.
static int static_tape_ptr(int dev, cudaStream_t st, double** out) {
    if (dev < 0 || dev >= 64) return fail(nullptr, DR_ERR_CUDA, "device ordinal %d out of range", dev);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return fail(nullptr, DR_ERR_CUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (cs == cudaStreamCaptureStatusNone || !g_static_ready[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_tape);
        if (e != cudaSuccess) return fail(nullptr, DR_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_static_tape_ptr[dev] = reinterpret_cast<double*>(p);
        g_static_ready[dev] = true;
    }
    *out = g_static_tape_ptr[dev];
    return DR_OK;
}

extern "C" int dr_slope_gradient_static(const dr_static_args* s) {
    if (!s) return fail(nullptr, DR_ERR_ARG, "dr_slope_gradient_static: args is NULL");
    if (s->L < 1 || s->L > DR_MAXL) return fail(nullptr, DR_ERR_SHAPE, "L = %d outside 1..%d", s->L, DR_MAXL);
    if (!s->W || !s->b || !s->A || !s->B || !s->lo || !s->hi || !s->alpha || !s->dalpha)
        return fail(nullptr, DR_ERR_ARG, "dr_slope_gradient_static: NULL device pointer");
    if (s->D < 0 || s->H < 1) return fail(nullptr, DR_ERR_ARG, "D = %lld, H = %d", (long long)s->D, s->H);
    if (!(s->margin_rho >= 0.0) || s->margin_rho > 1e-2) return fail(nullptr, DR_ERR_ARG, "margin_rho %g", s->margin_rho);
    NetDesc N{};
    N.L = s->L;
    N.maxw = 0;
    int64_t nw = 0, nb = 0;
    for (int l = 0; l <= s->L; ++l) {
        if (s->widths[l] < 1 || s->widths[l] > 4096) return fail(nullptr, DR_ERR_SHAPE, "width[%d] = %d", l, s->widths[l]);
        N.w[l] = s->widths[l];
        if (l >= 1) N.maxw = std::max(N.maxw, s->widths[l]);
    }
    for (int l = 1; l < s->L; ++l) {
        N.hoff[l] = N.hidden;
        N.hidden += N.w[l];
    }
    N.hoff[s->L] = N.hidden;
    for (int l = 0; l < s->L; ++l) {
        N.Woff[l] = nw;
        N.boff[l] = nb;
        nw += (int64_t)N.w[l + 1] * N.w[l];
        nb += N.w[l + 1];
    }
    N.n = N.w[0];
    N.m = N.w[s->L];
    N.H = s->H;
    if (N.n > 64 || N.m > 64) return fail(nullptr, DR_ERR_SHAPE, "n = %d, m = %d (supported 1..64)", N.n, N.m);
    const double need = (double)s->D * s->H * tape_stride(N) * sizeof(double);
    if (need > (double)DR_STATIC_SCRATCH_BYTES)
        return fail(nullptr, DR_ERR_SHAPE,
                    "dr_slope_gradient_static: needs %.0f bytes of scratch for D=%lld, H=%d, n=%d; the static limit is %u bytes",
                    need, (long long)s->D, s->H, N.n, (unsigned)DR_STATIC_SCRATCH_BYTES);
    const FusedLayout fwd = fused_layout(N, false), bwd = fused_layout(N, true);
    if (bwd.total > kMaxSmem) return fail(nullptr, DR_ERR_SHAPE, "controller too wide for the fused kernels");
    if (s->D == 0) return DR_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, DR_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s->stream);
    double* tape = nullptr;
    TRY(static_tape_ptr(dev, st, &tape));

    FusedArgs a;
    memset(&a, 0, sizeof(a));
    a.net = N;
    a.W = s->W;
    a.b = s->b;
    a.A = s->A;
    a.B = s->B;
    a.e = s->e;
    a.lo0 = s->lo;
    a.hi0 = s->hi;
    a.alpha = s->alpha;
    a.mode = DR_SLOPE_USER_K;
    a.rho = (float)s->margin_rho;
    a.box_margin = std::ldexp(1.0, -18);
    a.V = s->V;
    a.tape = tape;
    a.tape_stride = tape_stride(N);
    a.dalpha = s->dalpha;
    const int nt = fused_threads(N);
    const int64_t chunk = 1 << 20;
    for (int pass = 0; pass < 2; ++pass) {
        a.lay = pass == 0 ? fwd : bwd;
        const int smem = a.lay.total;
        for (int64_t d0 = 0; d0 < s->D; d0 += chunk) {
            a.d0 = d0;
            const unsigned nd = (unsigned)std::min(chunk, s->D - d0);
            if (pass == 0 && nt == 128) {
                CUDA_TRY(nullptr, cudaFuncSetAttribute(k_fused_forward<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                k_fused_forward<128><<<nd, 128, smem, st>>>(a);
            } else if (pass == 0) {
                CUDA_TRY(nullptr, cudaFuncSetAttribute(k_fused_forward<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                k_fused_forward<256><<<nd, 256, smem, st>>>(a);
            } else if (nt == 128) {
                CUDA_TRY(nullptr, cudaFuncSetAttribute(k_fused_backward<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                k_fused_backward<128><<<nd, 128, smem, st>>>(a);
            } else {
                CUDA_TRY(nullptr, cudaFuncSetAttribute(k_fused_backward<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                k_fused_backward<256><<<nd, 256, smem, st>>>(a);
            }
            CUDA_TRY(nullptr, cudaGetLastError());
        }
        a.V = nullptr;
    }
    return DR_OK;
}
