// Shared device-side definitions of the reachability kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define DR_MAXL 8  // maximum number of affine layers of the controller

// Shape of the controller/dynamics, passed by value to every kernel.
struct NetDesc {
    int L;                   // affine layers
    int n, m, H;             // state dim, control dim, horizon
    int hidden;              // n_1 + ... + n_{L-1}
    int w[DR_MAXL + 1];      // widths n_0 .. n_L
    int hoff[DR_MAXL + 1];   // hoff[l] = offset of hidden layer l (1-based) in the concatenated hidden vector
    int64_t Woff[DR_MAXL];   // offset of layer l+1's weights in the packed weight array (floats)
    int64_t boff[DR_MAXL];   // offset of layer l+1's biases in the packed bias array
    int maxw;                // max over n_1..n_L
};

// Per-domain split record as uploaded: (t, layer, neuron, sign).
struct SplitRec {
    int t, layer, neuron, sign;
};

__device__ __forceinline__ float posf(float x) { return x > 0.f ? x : 0.f; }

// A running sum of FP32 terms kept as an unevaluated pair hi + lo: each term enters by TwoSum
// (Knuth; error-free), so the pair holds the sum to about 2^-48 of its magnitude with FP32 adds only.
// Summing FP32 partials this way and converting once replaces an FP64 conversion and add per term;
// on a GPU whose FP64 rate is a small fraction of its FP32 rate that is the cheaper way to the same
// FP64 value (the FP64 sum rounds to 2^-53 per add; both are far inside the outward margins).
struct F32Pair {
    float hi = 0.f, lo = 0.f;
};
__device__ __forceinline__ void pair_add(F32Pair& p, float x) {
    const float s = __fadd_rn(p.hi, x);
    const float bp = __fsub_rn(s, p.hi);
    const float e = __fadd_rn(__fsub_rn(p.hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    p.hi = s;
    p.lo = __fadd_rn(p.lo, e);
}
// The pair's value in FP64; a non-finite running sum (an infinite or NaN term, or FP32 overflow)
// is returned as it is, so it stays non-finite (and is flagged downstream) rather than turning NaN.
__device__ __forceinline__ double pair_value(const F32Pair& p) {
    return isfinite(p.hi) ? (double)p.hi + (double)p.lo : (double)p.hi;
}
__device__ __forceinline__ float negf(float x) { return x < 0.f ? x : 0.f; }
__device__ __forceinline__ double posd(double x) { return x > 0.0 ? x : 0.0; }
__device__ __forceinline__ double negd(double x) { return x < 0.0 ? x : 0.0; }
__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }
__device__ __forceinline__ double sgnd(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// odd leading dimension for shared-memory matrices (row-parallel access is bank-conflict free)
__host__ __device__ __forceinline__ int odd_ld(int x) { return x | 1; }

#define DR_STATUS_NONFINITE_BIT 1u
#define DR_STATUS_INFEASIBLE_BIT 2u
#define DR_STATUS_MARGIN_BIT 4u

// The default outward box margin is calibrated on passes whose rows' summed term magnitudes S stay
// within this factor of the Taylor model's scale max_i (|c_i| + sum_k |P_ik| + max |I_i|) (measured:
// at most 18 on the workloads and 126 with first-layer biases shifted by +-6; 362 and more with
// shifts of +-50, where the margin no longer covers the FP32 rounding).  A row beyond it raises
// DR_STATUS_MARGIN_BIT.
#define DR_MARGIN_RATIO 256.0f

// max_i (|c_i| + sum_k |P_ik| + max(|Ilo_i|, |Ihi_i|)) of an FP64 Taylor model, as FP32.
__device__ __forceinline__ float tm_scale(const double* c, const double* P, const double* Ilo, const double* Ihi, int n) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) {
        float r = fabsf((float)c[i]) + fmaxf(fabsf((float)Ilo[i]), fabsf((float)Ihi[i]));
        for (int k = 0; k < n; ++k) r += fabsf((float)P[i * n + k]);
        s = fmaxf(s, r);
    }
    return s;
}

#define DR_SLOPE_ADAPTIVE_K 0
#define DR_SLOPE_CHORD_K 1
#define DR_SLOPE_ZERO_K 2
#define DR_SLOPE_USER_K 3
