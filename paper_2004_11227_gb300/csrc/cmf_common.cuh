// Shared device helpers of libcmf: storage types, projections, coefficient
// bundles and the launch-error plumbing.  Everything here is float32
// arithmetic on values stored as float32 / float16 / bfloat16.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "../../include/cmf.h"

namespace cmf {

// ---- storage types -------------------------------------------------------

template <typename S> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float ldw(const float* p) { return *p; }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
    static __device__ __forceinline__ float rt(float v) { return v; }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float ldw(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ float rt(float v) {
        return __half2float(__float2half_rn(v));
    }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) {
        return __bfloat162float(__ldg(p));
    }
    static __device__ __forceinline__ float ldw(const __nv_bfloat16* p) {
        return __bfloat162float(*p);
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) {
        *p = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ float rt(float v) {
        return __bfloat162float(__float2bfloat16_rn(v));
    }
};

inline size_t dtype_size(int storage) { return storage == CMF_F32 ? 4 : 2; }

// ---- per-device memo of launch-configuration queries ----------------------
// Function attributes (a raised shared-memory limit) and occupancy belong to
// a device, so a launcher that caches them keeps one entry per device
// ordinal.  compute(dev, v) runs with that device current and fills v (> 0);
// entries are atomics, so concurrent host threads at worst compute one twice.
constexpr int kMaxDevices = 64;
template <typename F>
inline cudaError_t per_device(std::atomic<long long> (&memo)[kMaxDevices], F compute,
                              long long& out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool slot = dev >= 0 && dev < kMaxDevices;
    if (slot) {
        const long long v = memo[dev].load(std::memory_order_acquire);
        if (v > 0) {
            out = v;
            return cudaSuccess;
        }
    }
    long long v = 0;
    if ((e = compute(dev, v)) != cudaSuccess) return e;
    if (slot && v > 0) memo[dev].store(v, std::memory_order_release);
    out = v;
    return cudaSuccess;
}

// Raise `kern`'s dynamic shared-memory limit on the current device to at
// least dyn bytes.  memo (the caller's per-kernel table) holds the limit set
// on each device; one lock orders the raises, so a smaller request never
// lowers a limit a concurrent call has just raised.
inline std::mutex& attr_mutex() {
    static std::mutex m;
    return m;
}
template <typename Kern>
inline cudaError_t raise_dyn_smem(std::atomic<long long> (&memo)[kMaxDevices], Kern kern,
                                  size_t dyn) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool slot = dev >= 0 && dev < kMaxDevices;
    if (slot && memo[dev].load(std::memory_order_acquire) >= (long long)dyn) return cudaSuccess;
    std::lock_guard<std::mutex> lock(attr_mutex());
    if (slot && memo[dev].load(std::memory_order_acquire) >= (long long)dyn) return cudaSuccess;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)) !=
        cudaSuccess)
        return e;
    if (slot) memo[dev].store((long long)dyn, std::memory_order_release);
    return cudaSuccess;
}

// ---- pointwise projections (Eq. projections) -----------------------------

// P_alpha: q / max(1, |q|/alpha); alpha <= 0 gives 0.  Anisotropic option:
// clamp each component to [-alpha, alpha].
template <bool ANISO>
__device__ __forceinline__ void project_alpha(float& x, float& y, float al) {
    al = fmaxf(al, 0.0f);
    if (ANISO) {
        x = fminf(fmaxf(x, -al), al);
        y = fminf(fmaxf(y, -al), al);
    } else {
        float n2 = x * x + y * y;
        if (n2 > al * al) {
            float s = al * rsqrtf(n2);
            x *= s;
            y *= s;
        }
    }
}

// ---- alpha: a plane or a constant ----------------------------------------

struct Alpha {
    const float* plane;  // NULL => constant
    float value;
    __device__ __forceinline__ float at(size_t k) const {
        return plane ? __ldg(plane + k) : value;
    }
};

// ---- grid geometry -------------------------------------------------------

struct Grid {
    int H, W, pitch;
    size_t plane;  // H * pitch
    __device__ __forceinline__ size_t idx(int r, int c) const {
        return (size_t)r * (size_t)pitch + (size_t)c;
    }
};

// ---- ADMM coefficients (float32, precomputed on the host) ----------------
// One formula covers rpADMMII (Eckstein-Bertsekas) and rpADMMI/pADMMI
// (Fortin-Glowinski):
//   p update uses rho_p (= rho for EB, 1 for FG),
//   u <- u - cu * ((Ap)^{k+1} - omr * (Ap)^k + rho_p * div q^{k+1})
// with cu = c, omr = 1 - rho for EB and cu = r c, omr = 0 for FG.
struct AdmmCoef {
    float inv_a;     // 1/a
    float inv_c;     // 1/c
    float rho_p;     // rho (EB) or 1 (FG)
    float rho_a1;    // rho_p / a1
    float inv_a1;    // 1 / a1
    float inv_a2;    // 1 / a2 (Potts)
    float cu;        // c (EB, TY) or r c (FG)
    float omr;       // 1 - rho (EB) or 0 (FG, TY)
    float inv_L;     // 1 / L (Potts pADMM-TY)
    int ty;          // 1: pADMM-TY sequential p-steps (Eq. ADMM:Tai_yuan)
    // ALG1 (Chambolle-Pock, Eq. iteration:pd:seg / Eq. alg1:4labels) runs in
    // the same kernels: with inv_c = 1/tau the source field g equals
    // -ubar/tau, where ubar = u - tau (div q + p_t - p_s) = 2u^k - u^{k-1} is
    // the extrapolated multiplier, so the q-step q - sigma grad ubar is the
    // ADMM q-step with inv_a = sigma tau; cu = tau.
    int cp;          // 1: ALG1 dual steps on p with ubar = -tau g
    float sigma;     // ALG1 dual step size
    float tau;       // ALG1 primal step size
};

// Pointwise p / u step of the binary ADMM family, rounded to the storage
// type.  rpADMMII / rpADMMI (Eq. rpADMMII, Eq. rpADMMI): p_t and p_s both
// read p^k (Jacobi), then the multiplier update.  pADMM-TY (Eq.
// ADMM:Tai_yuan): p_s from p_t^k, then p_t from p_s^{k+1}, then u.  ALG1
// (Eq. iteration:pd:seg): p_t, p_s ascend along ubar = -tau g (g: this
// pixel's source field of the iteration), then u descends.
template <typename S>
__device__ __forceinline__ void binary_pu(const AdmmCoef& K, float g, float d, float ps0,
                                          float pt0, float u0, float cs, float ct, float& ps1,
                                          float& pt1, float& u1) {
    using St = Store<S>;
    if (K.cp) {
        const float ub = -K.tau * g;
        pt1 = St::rt(fminf(pt0 + K.sigma * ub, ct));
        ps1 = St::rt(fminf(ps0 - K.sigma * ub + K.sigma, cs));
        u1 = u0 - K.tau * (d + pt1 - ps1);
    } else if (K.ty) {
        ps1 = St::rt(fminf(pt0 + d - u0 * K.inv_c + K.inv_c, cs));
        pt1 = St::rt(fminf(ps1 - d + u0 * K.inv_c, ct));
        u1 = u0 - K.cu * (pt1 - ps1 + d);
    } else {
        pt1 = St::rt(fminf(pt0 - K.rho_a1 * (pt0 - ps0) + K.inv_a1 * (-K.rho_p * d + u0 * K.inv_c),
                           ct));
        ps1 = St::rt(fminf(ps0 - K.rho_a1 * (ps0 - pt0) +
                               K.inv_a1 * (K.rho_p * d - u0 * K.inv_c + K.inv_c),
                           cs));
        u1 = u0 - K.cu * ((pt1 - ps1) - K.omr * (pt0 - ps0) + K.rho_p * d);
    }
}

// Potts, one label of one pixel: p_i^{k+1} (rounded), the label's share of
// the p_s update (acc_a, acc_b) and v_i with u_i^{k+1} = v_i + cu p_s^{k+1}.
// rpADMMII / rpADMMI: Eqs. after Thm 2 / Eq. multi:fg:4; pADMM-TY: Eq.
// mADMM:Tai_yuan with p_s from the new p_i; ALG1: Eq. alg1:4labels with
// ubar_i = -tau g (g: this label's source field at the pixel).
template <typename S>
__device__ __forceinline__ float potts_label_pu(const AdmmCoef& K, float g, float d, float p0,
                                                float ps0, float u0, float cl, float& acc_a,
                                                float& acc_b, float& v) {
    using St = Store<S>;
    float p1;
    if (K.cp) {
        const float ub = -K.tau * g;
        p1 = St::rt(fminf(p0 + K.sigma * ub, cl));
        acc_a += ub;
        v = u0 - K.tau * (d + p1);
    } else if (K.ty) {
        p1 = St::rt(fminf(ps0 - d + u0 * K.inv_c, cl));
        acc_a += p1 + d - u0 * K.inv_c;
        v = u0 - K.cu * (p1 + d);
    } else {
        p1 = St::rt(fminf(p0 - (K.rho_p * (p0 - ps0) - u0 * K.inv_c + K.rho_p * d) * K.inv_a1, cl));
        acc_a += K.rho_p * d;
        acc_b += K.rho_p * (p0 - ps0) - u0 * K.inv_c;
        v = u0 - K.cu * (p1 - K.omr * (p0 - ps0) + K.rho_p * d);
    }
    return p1;
}

// p_s^{k+1} from the accumulated label terms.  The Potts p_s plane is stored
// as float32 whatever the flow storage: one plane per pixel (4 bytes more per
// pixel and iteration than 16-bit), and its rounding to 16 bits alone holds
// the certified gap of the 16-label workload near 4e-4.
__device__ __forceinline__ float potts_ps_update(const AdmmCoef& K, float ps0, float acc_a,
                                                 float acc_b) {
    if (K.cp) return ps0 - K.sigma * (acc_a + acc_b) + K.sigma;
    return K.ty ? (acc_a + K.inv_c) * K.inv_L : ps0 + (acc_a + acc_b + K.inv_c) * K.inv_a2;
}

// ---- DR coefficients -----------------------------------------------------
struct DrCoef {
    float sigma, tau, rho;
    float inv_st;    // 1 / (sigma tau)
    float kappa;     // 2 (binary) or L + 1 (Potts)
    float Lm1;       // L - 1 (Potts)
    int sweeps;
};

// rPDRQ flow steps and reflections of one pixel (Eq. iteration:quadratic:seg):
// q = qbar - tau grad u, p_t = pbar_t + tau u, p_s = pbar_s - tau u, then
// qbar += rho (P_alpha(2q - qbar) - q), pbar_t += rho (min(2p_t - pbar_t, C_t)
// - p_t), pbar_s += rho (min(2p_s - pbar_s + tau, C_s) - p_s).
template <typename S, bool ANISO>
__device__ __forceinline__ void binary_dr_flows(const DrCoef& D, float uc, float gx, float gy,
                                                float qbx, float qby, float pbs, float pbt,
                                                float al, float cs, float ct, float& oqx,
                                                float& oqy, float& ops, float& opt) {
    const float q1 = qbx - D.tau * gx, q2 = qby - D.tau * gy;
    float tx = 2.f * q1 - qbx, ty = 2.f * q2 - qby;
    project_alpha<ANISO>(tx, ty, al);
    oqx = qbx + D.rho * (tx - q1);
    oqy = qby + D.rho * (ty - q2);
    const float pt1 = pbt + D.tau * uc, ps1 = pbs - D.tau * uc;
    opt = pbt + D.rho * (fminf(2.f * pt1 - pbt, ct) - pt1);
    ops = pbs + D.rho * (fminf(2.f * ps1 - pbs + D.tau, cs) - ps1);
}


AdmmCoef make_admm_coef(const cmf_params& p, int L);
DrCoef make_dr_coef(const cmf_params& p, int L, bool potts);

}  // namespace cmf

#define CMF_CUDA_TRY(expr)                                       \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) return CMF_ECUDA;                 \
    } while (0)
