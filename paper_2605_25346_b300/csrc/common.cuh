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
__device__ __forceinline__ float negf(float x) { return x < 0.f ? x : 0.f; }
__device__ __forceinline__ double posd(double x) { return x > 0.0 ? x : 0.0; }
__device__ __forceinline__ double negd(double x) { return x < 0.0 ? x : 0.0; }
__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }
__device__ __forceinline__ double sgnd(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// odd leading dimension for shared-memory matrices (row-parallel access is bank-conflict free)
__host__ __device__ __forceinline__ int odd_ld(int x) { return x | 1; }

#define DR_STATUS_NONFINITE_BIT 1u
#define DR_STATUS_INFEASIBLE_BIT 2u

#define DR_SLOPE_ADAPTIVE_K 0
#define DR_SLOPE_CHORD_K 1
#define DR_SLOPE_ZERO_K 2
#define DR_SLOPE_USER_K 3
