// Shared pieces of the warp-strip kernels (cmf_potts_strip.cu,
// cmf_binary_strip.cu): a warp owns a strip of 64 columns, two adjacent
// columns per lane, and streams down a band of rows.
#pragma once

#include "cmf_common.cuh"

namespace cmf {
namespace strip {

constexpr int kStripOut = 60;   // output columns per warp strip
constexpr int kStripWarps = 4;  // warps per block

// Two adjacent elements of a plane: raw pair type and conversions.
template <typename S>
struct Pair;
template <>
struct Pair<float> {
    using T = float2;
    static __device__ __forceinline__ T ld(const float* p) {
        return __ldg(reinterpret_cast<const float2*>(p));
    }
    // read once in this launch: evict-first in L1 and L2 (ld.global.cs)
    static __device__ __forceinline__ T ldcs(const float* p) {
        return __ldcs(reinterpret_cast<const float2*>(p));
    }
    static __device__ __forceinline__ void stcs(float* p, float a, float b) {
        __stcs(reinterpret_cast<float2*>(p), make_float2(a, b));
    }
    static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ float2 f2(T v) { return v; }
    static __device__ __forceinline__ void st(float* p, float a, float b) {
        *reinterpret_cast<float2*>(p) = make_float2(a, b);
    }
    // the pair as a store followed by a load would give it
    static __device__ __forceinline__ T pk(float a, float b) { return make_float2(a, b); }
};
template <>
struct Pair<__half> {
    using T = __half2;
    static __device__ __forceinline__ T ld(const __half* p) {
        return __ldg(reinterpret_cast<const __half2*>(p));
    }
    static __device__ __forceinline__ T ldcs(const __half* p) {
        return __ldcs(reinterpret_cast<const __half2*>(p));
    }
    static __device__ __forceinline__ void stcs(__half* p, float a, float b) {
        __stcs(reinterpret_cast<__half2*>(p), __floats2half2_rn(a, b));
    }
    static __device__ __forceinline__ T zero() { return __float2half2_rn(0.f); }
    static __device__ __forceinline__ float2 f2(T v) { return __half22float2(v); }
    static __device__ __forceinline__ void st(__half* p, float a, float b) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
    }
    static __device__ __forceinline__ T pk(float a, float b) { return __floats2half2_rn(a, b); }
};
template <>
struct Pair<__nv_bfloat16> {
    using T = __nv_bfloat162;
    static __device__ __forceinline__ T ld(const __nv_bfloat16* p) {
        return __ldg(reinterpret_cast<const __nv_bfloat162*>(p));
    }
    static __device__ __forceinline__ T ldcs(const __nv_bfloat16* p) {
        return __ldcs(reinterpret_cast<const __nv_bfloat162*>(p));
    }
    static __device__ __forceinline__ void stcs(__nv_bfloat16* p, float a, float b) {
        __stcs(reinterpret_cast<__nv_bfloat162*>(p), __floats2bfloat162_rn(a, b));
    }
    static __device__ __forceinline__ T zero() { return __float2bfloat162_rn(0.f); }
    static __device__ __forceinline__ float2 f2(T v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float a, float b) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
    }
    static __device__ __forceinline__ T pk(float a, float b) {
        return __floats2bfloat162_rn(a, b);
    }
};

// P_alpha without a branch (Eq. projections): the scale is selected, so the
// reciprocal square root of a zero norm is computed and discarded.
template <bool ANISO>
__device__ __forceinline__ void project_sel(float& x, float& y, float al) {
    al = fmaxf(al, 0.0f);
    if (ANISO) {
        x = fminf(fmaxf(x, -al), al);
        y = fminf(fmaxf(y, -al), al);
    } else {
        const float n2 = x * x + y * y;
        const float s = n2 > al * al ? al * rsqrtf(n2) : 1.0f;
        x *= s;
        y *= s;
    }
}

// Warps of `kern` resident on the whole current device, for blocks of WPB
// warps with `dyn` bytes of dynamic shared memory (with dyn > 0 the kernel's
// dynamic shared-memory limit is raised to dyn first).  `memo` is the
// caller's per-kernel table: the queries run once per device.
template <int WPB = kStripWarps, typename Kern>
inline cudaError_t device_resident_warps(std::atomic<long long> (&memo)[kMaxDevices], Kern kern,
                                         size_t dyn, long long& out) {
    return per_device(
        memo,
        [&](int dev, long long& v) -> cudaError_t {
            cudaError_t e;
            if (dyn && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)dyn)) != cudaSuccess)
                return e;
            int sms = 0, blocks = 0;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) !=
                cudaSuccess)
                return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, WPB * 32,
                                                                    dyn)) != cudaSuccess)
                return e;
            v = (long long)sms * (blocks > 0 ? blocks : 1) * WPB;
            return cudaSuccess;
        },
        out);
}

// As device_resident_warps without dynamic shared memory; 0 when a query
// fails (the certificate launchers then size bands for their own grid).
template <typename Kern>
inline long long resident_warps(std::atomic<long long> (&memo)[kMaxDevices], Kern kern) {
    long long v = 0;
    return device_resident_warps(memo, kern, 0, v) == cudaSuccess ? v : 0;
}

// Band height for a grid: the fewest rounds of work items over the resident
// warps, each round costing its rows plus `halo` rows; ties go to taller bands.
inline int choose_rows(int H, int nstrips, long long resident, int rmin, int rmax, int halo) {
    int best_r = rmax;
    long long best_cost = -1;
    for (int r = rmin; r <= rmax; ++r) {
        const long long items = (long long)nstrips * ((H + r - 1) / r);
        const long long rounds = (items + resident - 1) / resident;
        const long long cost = rounds * (r + halo);
        if (best_cost < 0 || cost <= best_cost) {
            best_cost = cost;
            best_r = r;
        }
    }
    return best_r;
}

}  // namespace strip
}  // namespace cmf
