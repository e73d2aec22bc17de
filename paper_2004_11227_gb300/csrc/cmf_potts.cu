// Potts continuous max-flow kernels (Eq. potts-mf, L labels): cold start,
// rpADMMI / rpADMMII / pADMMI iterations (Eq. multi:fg:4 and the
// Eckstein-Bertsekas equations after Thm 2), rPDRQ iterations
// (Eq. pdrq:4labels for general L) and the FP64-accumulated certificates.
//
// Label planes are stacked [L][H][pitch].  A fused block walks all L labels
// of its tile, because p_s couples the labels of a pixel.
#include "cmf_kernels.cuh"

namespace cmf {

#define POTTS_PIXEL_PROLOGUE                                  \
    const Grid G = P.g;                                       \
    const int c = blockIdx.x * 32 + threadIdx.x;              \
    const int r = blockIdx.y * 8 + threadIdx.y;               \
    if (r >= G.H || c >= G.W) return;                         \
    const size_t k = G.idx(r, c);

// First cheapest label at plane offset k (ties to the lowest index).
__device__ __forceinline__ int argmin_label(const PottsProblem& P, size_t k, float& m) {
    int best = 0;
    m = potts_cost(P, 0, k);
    for (int i = 1; i < P.L; ++i) {
        const float v = potts_cost(P, i, k);
        if (v < m) {
            m = v;
            best = i;
        }
    }
    return best;
}

// ---------------------------------------------------------------------------
// Cold start: u_i = 1 for the cheapest label, q_i = 0, p_i = p_s = min_j C_j;
// rPDRQ stores ybar = y - tau K u: qbar_i = tau grad u_i,
// pbar_i = p_i - tau u_i, pbar_s = p_s + tau (sum_i u_i = 1).
// ---------------------------------------------------------------------------
template <typename S, bool DR>
__global__ void k_potts_init(PottsProblem P, PottsState<S> s, float tau) {
    POTTS_PIXEL_PROLOGUE
    using St = Store<S>;
    const size_t pl = G.plane;
    float m, mr, md;
    const int best = argmin_label(P, k, m);
    int bestr = -1, bestd = -1;
    if (DR && c < G.W - 1) bestr = argmin_label(P, k + 1, mr);
    if (DR && r < G.H - 1) bestd = argmin_label(P, k + G.pitch, md);
    for (int i = 0; i < P.L; ++i) {
        const size_t ki = i * pl + k;
        const float u = i == best ? 1.f : 0.f;
        float qx = 0.f, qy = 0.f, p = m;
        if (DR) {
            if (bestr >= 0) qx = tau * ((i == bestr ? 1.f : 0.f) - u);
            if (bestd >= 0) qy = tau * ((i == bestd ? 1.f : 0.f) - u);
            p = m - tau * u;
        }
        s.u[ki] = u;
        St::st(s.qx + ki, qx);
        St::st(s.qy + ki, qy);
        St::st(s.p + ki, p);
    }
    s.ps[k] = DR ? m + tau : m;
}

// ---------------------------------------------------------------------------
// The state of one storage type written into float32 planes (the switch of a
// two-phase solve from 16-bit to float32 storage): every value is exact in
// float32, so the iteration continues from the same state.
// ---------------------------------------------------------------------------
template <typename S>
__global__ void k_potts_widen(Grid G, int L, PottsState<S> a, PottsState<float> b) {
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int r = blockIdx.y * 8 + threadIdx.y;
    if (r >= G.H || c >= G.W) return;
    const size_t k = G.idx(r, c);
    for (int i = 0; i < L; ++i) {
        const size_t ki = (size_t)i * G.plane + k;
        b.u[ki] = a.u[ki];
        b.qx[ki] = Store<S>::ld(a.qx + ki);
        b.qy[ki] = Store<S>::ld(a.qy + ki);
        b.p[ki] = Store<S>::ld(a.p + ki);
    }
    b.ps[k] = a.ps[k];
}

// ---------------------------------------------------------------------------
// Fused ADMM iteration.  Per label i the tile computes
//   g_i = div q_i^k + p_i^k - p_s^k - u_i^k / c            (halo of 1)
//   q_i^{k+1} = P_alpha(q_i^k + (1/a) grad g_i)
//   d_i = div q_i^{k+1}
//   p_i^{k+1} = min(p_i - (rho_p (p_i - p_s) - u_i/c + rho_p d_i)/a1, C_i)
// and accumulates the p_s terms sum rho_p d_i + rho_p (p_i - p_s) - u_i/c.
// The multiplier update splits as u_i^{k+1} = v_i + cu p_s^{k+1} with
//   v_i = u_i - cu (p_i^{k+1} - omr (p_i^k - p_s^k) + rho_p d_i),
// so v_i is kept in shared memory until p_s^{k+1} is known.
// ---------------------------------------------------------------------------
template <typename S, bool ANISO, int ROWS>
__device__ __forceinline__ void potts_admm_tile(PottsProblem P, PottsState<S> s0, PottsState<S> s1, AdmmCoef K, int bx_, int by_) {
    constexpr int TX = 32, TY = 8 * ROWS;
    constexpr int GX = TX + 2, GY = TY + 2;
    constexpr int QX = TX + 1, QY = TY + 1;
    __shared__ float ps_s[GY][GX];
    __shared__ float g_s[GY][GX];
    __shared__ float qx_s[QY][QX];
    __shared__ float qy_s[QY][QX];
    extern __shared__ float v_s[];  // [L][TY][TX]
    using St = Store<S>;
    const Grid G = P.g;
    const size_t pl = G.plane;
    const int x0 = bx_ * TX, y0 = by_ * TY;
    const int tid = threadIdx.y * 32 + threadIdx.x;

    for (int i = tid; i < GX * GY; i += 256) {
        const int ly = i / GX, lx = i - ly * GX;
        const int r = y0 - 1 + ly, c = x0 - 1 + lx;
        ps_s[ly][lx] = (r >= 0 && r < G.H && c >= 0 && c < G.W) ? __ldg(s0.ps + G.idx(r, c))
                                                                 : 0.f;
    }
    float accd[ROWS], accp[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) accd[j] = accp[j] = 0.f;

#pragma unroll 1
    for (int l = 0; l < P.L; ++l) {
        const size_t lo = (size_t)l * pl;
        const S* qx0 = s0.qx + lo;
        const S* qy0 = s0.qy + lo;
        __syncthreads();
        for (int i = tid; i < GX * GY; i += 256) {
            const int ly = i / GX, lx = i - ly * GX;
            const int r = y0 - 1 + ly, c = x0 - 1 + lx;
            float g = 0.f;
            if (r >= 0 && r < G.H && c >= 0 && c < G.W) {
                const size_t k = G.idx(r, c);
                float dv = 0.f;
                if (c < G.W - 1) dv += St::ld(qx0 + k);
                if (c > 0) dv -= St::ld(qx0 + k - 1);
                if (r < G.H - 1) dv += St::ld(qy0 + k);
                if (r > 0) dv -= St::ld(qy0 + k - G.pitch);
                g = dv + St::ld(s0.p + lo + k) - ps_s[ly][lx] - __ldg(s0.u + lo + k) * K.inv_c;
            }
            g_s[ly][lx] = g;
        }
        __syncthreads();
        for (int i = tid; i < QX * QY; i += 256) {
            const int ly = i / QX, lx = i - ly * QX;
            const int r = y0 - 1 + ly, c = x0 - 1 + lx;
            float tx = 0.f, ty = 0.f;
            if (r >= 0 && r < G.H && c >= 0 && c < G.W) {
                const size_t k = G.idx(r, c);
                const float gc = g_s[ly][lx];
                tx = St::ld(qx0 + k) + (c < G.W - 1 ? (g_s[ly][lx + 1] - gc) * K.inv_a : 0.f);
                ty = St::ld(qy0 + k) + (r < G.H - 1 ? (g_s[ly + 1][lx] - gc) * K.inv_a : 0.f);
                project_alpha<ANISO>(tx, ty, P.alpha.at(k));
                tx = St::rt(tx);
                ty = St::rt(ty);
                if (ly >= 1 && lx >= 1) {
                    St::st(s1.qx + lo + k, tx);
                    St::st(s1.qy + lo + k, ty);
                }
            }
            qx_s[ly][lx] = tx;
            qy_s[ly][lx] = ty;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
            const int r = y0 + ly, c = x0 + lx;
            float v = 0.f;
            if (r < G.H && c < G.W) {
                const size_t k = G.idx(r, c);
                float d = 0.f;
                if (c < G.W - 1) d += qx_s[ly + 1][lx + 1];
                if (c > 0) d -= qx_s[ly + 1][lx];
                if (r < G.H - 1) d += qy_s[ly + 1][lx + 1];
                if (r > 0) d -= qy_s[ly][lx + 1];
                const float ps0 = ps_s[ly + 1][lx + 1];
                const float p0 = St::ld(s0.p + lo + k);
                const float u0 = __ldg(s0.u + lo + k);
                const float p1 = potts_label_pu<S>(K, g_s[ly + 1][lx + 1], d, p0, ps0, u0,
                                                   potts_cost(P, l, k), accd[j], accp[j], v);
                St::st(s1.p + lo + k, p1);
            }
            v_s[(l * TY + ly) * TX + lx] = v;
        }
    }

    float ps1[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
        const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
        const int r = y0 + ly, c = x0 + lx;
        ps1[j] = 0.f;
        if (r < G.H && c < G.W) {
            const float ps0 = ps_s[ly + 1][lx + 1];
            ps1[j] = potts_ps_update(K, ps0, accd[j], accp[j]);
            s1.ps[G.idx(r, c)] = ps1[j];
        }
    }
#pragma unroll 1
    for (int l = 0; l < P.L; ++l) {
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
            const int r = y0 + ly, c = x0 + lx;
            if (r < G.H && c < G.W)
                s1.u[(size_t)l * pl + G.idx(r, c)] = v_s[(l * TY + ly) * TX + lx] + K.cu * ps1[j];
        }
    }
}

template <typename S, bool ANISO, int ROWS>
__global__ void __launch_bounds__(256)
    k_potts_admm_fused(PottsProblem P, PottsState<S> s0, PottsState<S> s1, AdmmCoef K) {
    potts_admm_tile<S, ANISO, ROWS>(P, s0, s1, K, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Plain ADMM: per label g, q, div kernels; then one pointwise kernel for
// p_i, p_s and u_i.
// ---------------------------------------------------------------------------
template <typename S>
__device__ __forceinline__ float div_plane(const Grid& G, const S* qx, const S* qy, int r, int c,
                                           size_t k) {
    using St = Store<S>;
    float v = 0.f;
    if (c < G.W - 1) v += St::ldw(qx + k);
    if (c > 0) v -= St::ldw(qx + k - 1);
    if (r < G.H - 1) v += St::ldw(qy + k);
    if (r > 0) v -= St::ldw(qy + k - G.pitch);
    return v;
}

template <typename S>
__global__ void k_potts_plain_g(PottsProblem P, PottsState<S> s, int l, float* g, AdmmCoef K) {
    POTTS_PIXEL_PROLOGUE
    using St = Store<S>;
    const size_t lo = (size_t)l * G.plane;
    g[k] = div_plane(G, s.qx + lo, s.qy + lo, r, c, k) + St::ldw(s.p + lo + k) -
           s.ps[k] - s.u[lo + k] * K.inv_c;
}

template <typename S, bool ANISO>
__global__ void k_potts_plain_q(PottsProblem P, PottsState<S> s, int l, const float* g,
                                AdmmCoef K) {
    POTTS_PIXEL_PROLOGUE
    using St = Store<S>;
    const size_t lo = (size_t)l * G.plane;
    const float gc = g[k];
    float tx = St::ldw(s.qx + lo + k) + (c < G.W - 1 ? (g[k + 1] - gc) * K.inv_a : 0.f);
    float ty = St::ldw(s.qy + lo + k) + (r < G.H - 1 ? (g[k + G.pitch] - gc) * K.inv_a : 0.f);
    project_alpha<ANISO>(tx, ty, P.alpha.at(k));
    St::st(s.qx + lo + k, tx);
    St::st(s.qy + lo + k, ty);
}

template <typename S>
__global__ void k_potts_plain_div(PottsProblem P, PottsState<S> s, int l, float* d) {
    POTTS_PIXEL_PROLOGUE
    const size_t lo = (size_t)l * G.plane;
    d[lo + k] = div_plane(G, s.qx + lo, s.qy + lo, r, c, k);
}

template <typename S>
__global__ void k_potts_plain_pu(PottsProblem P, PottsState<S> s, const float* g, const float* d,
                                 AdmmCoef K) {
    POTTS_PIXEL_PROLOGUE
    using St = Store<S>;
    const size_t pl = G.plane;
    const float ps0 = s.ps[k];
    // p_i^{k+1} and v_i per label (v_i parked in u_i), then p_s^{k+1}, then
    // u_i^{k+1} = v_i + cu p_s^{k+1}
    float acc_a = 0.f, acc_b = 0.f;
    for (int l = 0; l < P.L; ++l) {
        const size_t ki = l * pl + k;
        float v;
        const float p1 = potts_label_pu<S>(K, g[ki], d[ki], St::ldw(s.p + ki), ps0, s.u[ki],
                                           potts_cost(P, l, k), acc_a, acc_b, v);
        St::st(s.p + ki, p1);
        s.u[ki] = v;
    }
    const float ps1 = potts_ps_update(K, ps0, acc_a, acc_b);
    for (int l = 0; l < P.L; ++l) s.u[l * pl + k] += K.cu * ps1;
    s.ps[k] = ps1;
}

// ---------------------------------------------------------------------------
// rPDRQ (Eq. pdrq:4labels, general L).  State (u_i, qbar_i, pbar_i, pbar_s).
//   b_i = -sigma (div qbar_i + pbar_i - pbar_s) + sigma tau (L u_i - U),
//         U = sum_j u_j^k   ((L-1) u_i - sum_{j != i} u_j = L u_i - U)
//   u_i <- sRBGS on sigma tau ((L+1) I - Lap) u_i = b_i
//   qbar_i += rho (P_alpha(2 q_i - qbar_i) - q_i), q_i = qbar_i - tau grad u_i
//   pbar_i += rho (min(2 p_i - pbar_i, C_i) - p_i), p_i = pbar_i + tau u_i
//   pbar_s += rho ((2 p_s - pbar_s + tau) - p_s), p_s = pbar_s - tau sum u_i
// ---------------------------------------------------------------------------
template <typename S, bool ANISO, int ROWS, int SW>
__device__ __forceinline__ void potts_dr_tile(PottsProblem P, PottsState<S> s0, PottsState<S> s1, DrCoef D, int bx_, int by_) {
    constexpr int TX = 32, TY = 8 * ROWS;
    constexpr int NH = 2 * SW + 1;
    constexpr int UX = TX + 1 + 2 * NH, UY = TY + 1 + 2 * NH;
    constexpr int BX = UX - 2, BY = UY - 2;
    __shared__ float u_s[UY][UX];
    __shared__ float b_s[BY][BX];
    __shared__ float U_s[BY][BX];
    __shared__ float pbs_s[BY][BX];
    using St = Store<S>;
    const Grid G = P.g;
    const size_t pl = G.plane;
    const int x0 = bx_ * TX, y0 = by_ * TY;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int ux0 = x0 - NH, uy0 = y0 - NH;
    const float st_ = D.sigma * D.tau;

    for (int i = tid; i < BX * BY; i += 256) {
        const int ly = i / BX, lx = i - ly * BX;
        const int r = uy0 + 1 + ly, c = ux0 + 1 + lx;
        float U = 0.f, pbs = 0.f;
        if (r >= 0 && r < G.H && c >= 0 && c < G.W) {
            const size_t k = G.idx(r, c);
            for (int l = 0; l < P.L; ++l) U += __ldg(s0.u + (size_t)l * pl + k);
            pbs = __ldg(s0.ps + k);
        }
        U_s[ly][lx] = U;
        pbs_s[ly][lx] = pbs;
    }
    float usum[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) usum[j] = 0.f;

#pragma unroll 1
    for (int l = 0; l < P.L; ++l) {
        const size_t lo = (size_t)l * pl;
        __syncthreads();
        for (int i = tid; i < UX * UY; i += 256) {
            const int ly = i / UX, lx = i - ly * UX;
            const int r = uy0 + ly, c = ux0 + lx;
            u_s[ly][lx] = (r >= 0 && r < G.H && c >= 0 && c < G.W)
                              ? __ldg(s0.u + lo + G.idx(r, c))
                              : 0.f;
        }
        __syncthreads();
        for (int i = tid; i < BX * BY; i += 256) {
            const int ly = i / BX, lx = i - ly * BX;
            const int r = uy0 + 1 + ly, c = ux0 + 1 + lx;
            float b = 0.f;
            if (r >= 0 && r < G.H && c >= 0 && c < G.W) {
                const size_t k = G.idx(r, c);
                float dv = 0.f;
                if (c < G.W - 1) dv += St::ld(s0.qx + lo + k);
                if (c > 0) dv -= St::ld(s0.qx + lo + k - 1);
                if (r < G.H - 1) dv += St::ld(s0.qy + lo + k);
                if (r > 0) dv -= St::ld(s0.qy + lo + k - G.pitch);
                b = -D.sigma * (dv + St::ld(s0.p + lo + k) - pbs_s[ly][lx]) +
                    st_ * ((float)P.L * u_s[ly + 1][lx + 1] - U_s[ly][lx]);
            }
            b_s[ly][lx] = b;
        }
        __syncthreads();
#pragma unroll 1
        for (int s = 0; s < NH; ++s) {
            const int colour = s & 1;
            const int grow = NH - 1 - s;
            const int lo2 = NH - grow;
            const int ny = TY + 1 + 2 * grow, nx = TX + 1 + 2 * grow;
            for (int i = tid; i < nx * ny; i += 256) {
                const int ly = lo2 + i / nx, lx = lo2 + i % nx;
                const int r = uy0 + ly, c = ux0 + lx;
                if (((r + c) & 1) != colour || r < 0 || r >= G.H || c < 0 || c >= G.W) continue;
                float sum = 0.f;
                int nnb = 0;
                if (c > 0) { sum += u_s[ly][lx - 1]; ++nnb; }
                if (c < G.W - 1) { sum += u_s[ly][lx + 1]; ++nnb; }
                if (r > 0) { sum += u_s[ly - 1][lx]; ++nnb; }
                if (r < G.H - 1) { sum += u_s[ly + 1][lx]; ++nnb; }
                u_s[ly][lx] = (b_s[ly - 1][lx - 1] * D.inv_st + sum) / (D.kappa + (float)nnb);
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
            const int r = y0 + ly, c = x0 + lx;
            if (r < G.H && c < G.W) {
                const size_t k = G.idx(r, c);
                const float uc = u_s[NH + ly][NH + lx];
                const float gx = c < G.W - 1 ? u_s[NH + ly][NH + lx + 1] - uc : 0.f;
                const float gy = r < G.H - 1 ? u_s[NH + ly + 1][NH + lx] - uc : 0.f;
                const float qbx = St::ld(s0.qx + lo + k), qby = St::ld(s0.qy + lo + k);
                const float q1 = qbx - D.tau * gx, q2 = qby - D.tau * gy;
                float tx = 2.f * q1 - qbx, ty = 2.f * q2 - qby;
                project_alpha<ANISO>(tx, ty, P.alpha.at(k));
                const float pb = St::ld(s0.p + lo + k);
                const float p1 = pb + D.tau * uc;
                s1.u[lo + k] = uc;
                St::st(s1.qx + lo + k, qbx + D.rho * (tx - q1));
                St::st(s1.qy + lo + k, qby + D.rho * (ty - q2));
                St::st(s1.p + lo + k, pb + D.rho * (fminf(2.f * p1 - pb, potts_cost(P, l, k)) - p1));
                usum[j] += uc;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
        const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
        const int r = y0 + ly, c = x0 + lx;
        if (r < G.H && c < G.W) {
            const float pbs = pbs_s[ly + NH - 1][lx + NH - 1];
            const float ps1 = pbs - D.tau * usum[j];
            s1.ps[G.idx(r, c)] = pbs + D.rho * ((2.f * ps1 - pbs + D.tau) - ps1);
        }
    }
}

template <typename S, bool ANISO, int ROWS, int SW>
__global__ void __launch_bounds__(256)
    k_potts_dr_fused(PottsProblem P, PottsState<S> s0, PottsState<S> s1, DrCoef D) {
    potts_dr_tile<S, ANISO, ROWS, SW>(P, s0, s1, D, blockIdx.x, blockIdx.y);
}

// Plain rPDRQ pieces.
template <typename S>
__global__ void k_potts_plain_usum(PottsProblem P, PottsState<S> s, float* U) {
    POTTS_PIXEL_PROLOGUE
    float a = 0.f;
    for (int l = 0; l < P.L; ++l) a += s.u[(size_t)l * G.plane + k];
    U[k] = a;
}

template <typename S>
__global__ void k_potts_plain_dr_b(PottsProblem P, PottsState<S> s, int l, const float* U,
                                   float* b, DrCoef D) {
    POTTS_PIXEL_PROLOGUE
    using St = Store<S>;
    const size_t lo = (size_t)l * G.plane;
    b[k] = -D.sigma * (div_plane(G, s.qx + lo, s.qy + lo, r, c, k) + St::ldw(s.p + lo + k) -
                       s.ps[k]) +
           D.sigma * D.tau * ((float)P.L * s.u[lo + k] - U[k]);
}

template <typename S, bool ANISO>
__global__ void k_potts_plain_dr_flows(PottsProblem P, PottsState<S> s, int l, DrCoef D) {
    POTTS_PIXEL_PROLOGUE
    using St = Store<S>;
    const size_t lo = (size_t)l * G.plane;
    const float uc = s.u[lo + k];
    const float gx = c < G.W - 1 ? s.u[lo + k + 1] - uc : 0.f;
    const float gy = r < G.H - 1 ? s.u[lo + k + G.pitch] - uc : 0.f;
    const float qbx = St::ldw(s.qx + lo + k), qby = St::ldw(s.qy + lo + k);
    const float q1 = qbx - D.tau * gx, q2 = qby - D.tau * gy;
    float tx = 2.f * q1 - qbx, ty = 2.f * q2 - qby;
    project_alpha<ANISO>(tx, ty, P.alpha.at(k));
    St::st(s.qx + lo + k, qbx + D.rho * (tx - q1));
    St::st(s.qy + lo + k, qby + D.rho * (ty - q2));
    const float pb = St::ldw(s.p + lo + k);
    const float p1 = pb + D.tau * uc;
    St::st(s.p + lo + k, pb + D.rho * (fminf(2.f * p1 - pb, potts_cost(P, l, k)) - p1));
}

template <typename S>
__global__ void k_potts_plain_dr_ps(PottsProblem P, PottsState<S> s, DrCoef D) {
    POTTS_PIXEL_PROLOGUE
    using St = Store<S>;
    float a = 0.f;
    for (int l = 0; l < P.L; ++l) a += s.u[(size_t)l * G.plane + k];
    const float pbs = s.ps[k];
    const float ps1 = pbs - D.tau * a;
    s.ps[k] = pbs + D.rho * ((2.f * ps1 - pbs + D.tau) - ps1);
}

// ---------------------------------------------------------------------------
// Certificates.  ub(x) = projection of u(x) onto the simplex:
// ub_i = max(u_i - theta, 0), theta from Michelot's active-set iteration
// (drop entries <= theta, recompute theta = (sum_active - 1)/n_active).  The
// thresholds never decrease, so a dropped entry stays dropped and the active
// set of a pass is {i : u_i > theta}: each pass sums and counts it afresh (no
// set bookkeeping) and the iteration stops when the count no longer changes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float simplex_theta(const float* u, size_t pl, int L, size_t k) {
    float sum = 0.f;
    for (int i = 0; i < L; ++i) sum += u[i * pl + k];
    int n = L;
    float theta = (sum - 1.f) / (float)n;
    for (int it = 0; it < L; ++it) {
        float s = 0.f;
        int m = 0;
        for (int i = 0; i < L; ++i) {
            const float v = u[i * pl + k];
            if (v > theta) {
                s += v;
                ++m;
            }
        }
        if (m == n || m == 0) break;
        n = m;
        theta = (s - 1.f) / (float)n;
    }
    return theta;
}

template <typename S, bool DR>
__device__ __forceinline__ void potts_flow_at(const PottsProblem& P, const PottsState<S>& s,
                                              float tau, size_t lo, int r, int c, float& fx,
                                              float& fy) {
    using St = Store<S>;
    const Grid& G = P.g;
    const size_t k = lo + G.idx(r, c);
    fx = St::ldw(s.qx + k);
    fy = St::ldw(s.qy + k);
    if (DR) {
        const float uc = s.u[k];
        if (c < G.W - 1) fx -= tau * (s.u[k + 1] - uc);
        if (r < G.H - 1) fy -= tau * (s.u[k + G.pitch] - uc);
    }
}

template <typename S, bool ANISO, bool DR>
__device__ __forceinline__ void potts_eval_tile(PottsProblem P, PottsState<S> s, float tau, double* out3, int bx_, int by_) {
    using St = Store<S>;
    const Grid G = P.g;
    const size_t pl = G.plane;
    const int c = bx_ * 32 + threadIdx.x;
    DF accE = {0.f, 0.f}, accD = {0.f, 0.f}, accR = {0.f, 0.f};
    for (int j = 0; j < EVAL_ROWS; ++j) {
        const int r = (by_ * 8 + threadIdx.y) * EVAL_ROWS + j;
        if (r >= G.H || c >= G.W) continue;
        const size_t k = G.idx(r, c);
        const float al = P.alpha.at(k);
        const float th = simplex_theta(s.u, pl, P.L, k);
        const float thr = c < G.W - 1 ? simplex_theta(s.u, pl, P.L, k + 1) : 0.f;
        const float thd = r < G.H - 1 ? simplex_theta(s.u, pl, P.L, k + G.pitch) : 0.f;
        float usum = 0.f;
        for (int l = 0; l < P.L; ++l) usum += s.u[(size_t)l * pl + k];
        float fs = s.ps[k];
        if (DR) fs -= tau * usum;
        float e = 0.f, rr2 = 0.f, dmin = 3.402823466e38f;
        for (int l = 0; l < P.L; ++l) {
            const size_t lo = (size_t)l * pl;
            const float ub = fmaxf(s.u[lo + k] - th, 0.f);
            const float gx = c < G.W - 1 ? fmaxf(s.u[lo + k + 1] - thr, 0.f) - ub : 0.f;
            const float gy = r < G.H - 1 ? fmaxf(s.u[lo + k + G.pitch] - thd, 0.f) - ub : 0.f;
            const float tv = ANISO ? fabsf(gx) + fabsf(gy) : sqrtf(gx * gx + gy * gy);
            const float Cl = potts_cost(P, l, k);
            e += ub * Cl + al * tv;
            float fx, fy, fxl = 0.f, fyl = 0.f, fxu = 0.f, fyu = 0.f;
            potts_flow_at<S, DR>(P, s, tau, lo, r, c, fx, fy);
            if (c > 0) potts_flow_at<S, DR>(P, s, tau, lo, r, c - 1, fxl, fyl);
            if (r > 0) potts_flow_at<S, DR>(P, s, tau, lo, r - 1, c, fxu, fyu);
            float fp = St::ldw(s.p + lo + k);
            if (DR) fp += tau * s.u[lo + k];
            const float dv = (c < G.W - 1 ? fx : 0.f) - fxl + (r < G.H - 1 ? fy : 0.f) - fyu;
            const float rr = dv - fs + fp;
            rr2 += rr * rr;
            project_alpha<ANISO>(fx, fy, al);
            if (c > 0) project_alpha<ANISO>(fxl, fyl, P.alpha.at(k - 1));
            if (r > 0) project_alpha<ANISO>(fxu, fyu, P.alpha.at(k - G.pitch));
            const float dp = (c < G.W - 1 ? fx : 0.f) - fxl + (r < G.H - 1 ? fy : 0.f) - fyu;
            dmin = fminf(dmin, Cl + dp);
        }
        df_add(accE, e);
        df_add(accD, dmin);
        df_add(accR, rr2);
    }
    block_reduce3_store_df(accE, accD, accR, out3);
}

template <typename S, bool ANISO, bool DR>
__global__ void __launch_bounds__(256)
    k_potts_eval(PottsProblem P, PottsState<S> s, float tau, double* partials, EvalTail T) {
    potts_eval_tile<S, ANISO, DR>(P, s, tau, partials + 3 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x), blockIdx.x, blockIdx.y);
    eval_tail(T, partials, gridDim.x * gridDim.y);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static inline dim3 pgrid(const Grid& G, int rows_per_block) {
    return dim3((G.W + 31) / 32, (G.H + rows_per_block - 1) / rows_per_block);
}

template <typename S>
static cudaError_t potts_init_s(const PottsProblem& P, const PottsStateV& sv, bool dr, float tau,
                                cudaStream_t st) {
    const PottsState<S> s = sv.as<S>();
    if (dr) k_potts_init<S, true><<<pgrid(P.g, 8), dim3(32, 8), 0, st>>>(P, s, tau);
    else k_potts_init<S, false><<<pgrid(P.g, 8), dim3(32, 8), 0, st>>>(P, s, tau);
    return cudaGetLastError();
}

cudaError_t potts_widen(int storage, const Grid& G, int L, const PottsStateV& a,
                        const PottsStateV& b, cudaStream_t st) {
    const dim3 grid((G.W + 31) / 32, (G.H + 7) / 8);
    const PottsState<float> B = b.as<float>();
    switch (storage) {
        case CMF_F16:
            k_potts_widen<__half><<<grid, dim3(32, 8), 0, st>>>(G, L, a.as<__half>(), B);
            break;
        case CMF_BF16:
            k_potts_widen<__nv_bfloat16>
                <<<grid, dim3(32, 8), 0, st>>>(G, L, a.as<__nv_bfloat16>(), B);
            break;
        default:
            k_potts_widen<float><<<grid, dim3(32, 8), 0, st>>>(G, L, a.as<float>(), B);
    }
    return cudaGetLastError();
}

cudaError_t potts_init(int storage, const PottsProblem& P, const PottsStateV& s, bool dr,
                       float tau, cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return potts_init_s<float>(P, s, dr, tau, st);
        case CMF_F16: return potts_init_s<__half>(P, s, dr, tau, st);
        default: return potts_init_s<__nv_bfloat16>(P, s, dr, tau, st);
    }
}

template <typename S, bool ANISO, int ROWS>
static cudaError_t launch_potts_admm_fused(const PottsProblem& P, const PottsState<S>& a,
                                           const PottsState<S>& b, const AdmmCoef& K,
                                           cudaStream_t st) {
    const size_t dyn = (size_t)P.L * (8 * ROWS) * 32 * sizeof(float);
    auto kern = k_potts_admm_fused<S, ANISO, ROWS>;
    // static + dynamic shared memory above 48 KB needs the opt-in; raise the
    // limit per device to the largest request seen so far
    static std::atomic<long long> memo[kMaxDevices];
    {
        const cudaError_t e = raise_dyn_smem(memo, kern, dyn);
        if (e != cudaSuccess) return e;
    }
    kern<<<pgrid(P.g, 8 * ROWS), dim3(32, 8), dyn, st>>>(P, a, b, K);
    return cudaGetLastError();
}

template <typename S, bool ANISO>
static cudaError_t potts_admm_step_t(const PottsProblem& P, const PottsState<S>& a,
                                     const PottsState<S>& b, const AdmmCoef& K, bool plain,
                                     float* tmp, cudaStream_t st) {
    if (!plain) {
        if (P.L <= 8) return launch_potts_admm_fused<S, ANISO, 4>(P, a, b, K, st);
        if (P.L <= 16) return launch_potts_admm_fused<S, ANISO, 2>(P, a, b, K, st);
        return launch_potts_admm_fused<S, ANISO, 1>(P, a, b, K, st);
    }
    const dim3 gr = pgrid(P.g, 8), bl(32, 8);
    float* g = tmp;                        // L planes (ALG1 reads them back)
    float* d = tmp + P.L * P.g.plane;      // L planes
    for (int l = 0; l < P.L; ++l) {
        k_potts_plain_g<S><<<gr, bl, 0, st>>>(P, a, l, g + l * P.g.plane, K);
        k_potts_plain_q<S, ANISO><<<gr, bl, 0, st>>>(P, a, l, g + l * P.g.plane, K);
        k_potts_plain_div<S><<<gr, bl, 0, st>>>(P, a, l, d);
    }
    k_potts_plain_pu<S><<<gr, bl, 0, st>>>(P, a, g, d, K);
    return cudaGetLastError();
}

template <typename S, bool ANISO>
static cudaError_t potts_dr_step_t(const PottsProblem& P, const PottsState<S>& a,
                                   const PottsState<S>& b, const DrCoef& D, bool plain,
                                   float* tmp, cudaStream_t st) {
    if (!plain) {
        constexpr int ROWS = 4;
        const dim3 gr = pgrid(P.g, 8 * ROWS), bl(32, 8);
        switch (D.sweeps) {
            case 1: k_potts_dr_fused<S, ANISO, ROWS, 1><<<gr, bl, 0, st>>>(P, a, b, D); break;
            case 2: k_potts_dr_fused<S, ANISO, ROWS, 2><<<gr, bl, 0, st>>>(P, a, b, D); break;
            case 3: k_potts_dr_fused<S, ANISO, ROWS, 3><<<gr, bl, 0, st>>>(P, a, b, D); break;
            default: k_potts_dr_fused<S, ANISO, ROWS, 4><<<gr, bl, 0, st>>>(P, a, b, D); break;
        }
        return cudaGetLastError();
    }
    const dim3 gr = pgrid(P.g, 8), bl(32, 8);
    float* U = tmp;
    float* bb = tmp + P.g.plane;
    k_potts_plain_usum<S><<<gr, bl, 0, st>>>(P, a, U);
    for (int l = 0; l < P.L; ++l) {
        float* ul = a.u + (size_t)l * P.g.plane;
        k_potts_plain_dr_b<S><<<gr, bl, 0, st>>>(P, a, l, U, bb, D);
        cudaError_t e = halfsweeps(P.g, ul, bb, D, st);
        if (e != cudaSuccess) return e;
    }
    for (int l = 0; l < P.L; ++l) k_potts_plain_dr_flows<S, ANISO><<<gr, bl, 0, st>>>(P, a, l, D);
    k_potts_plain_dr_ps<S><<<gr, bl, 0, st>>>(P, a, D);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t potts_step_s(const PottsProblem& P, const PottsStateV& a,
                                const PottsStateV& b, const StepConfig& cfg, float* tmp,
                                cudaStream_t st) {
    const PottsState<S> A = a.as<S>(), B = b.as<S>();
    if (cfg.dr)
        return cfg.aniso ? potts_dr_step_t<S, true>(P, A, B, cfg.dc, cfg.plain, tmp, st)
                         : potts_dr_step_t<S, false>(P, A, B, cfg.dc, cfg.plain, tmp, st);
    return cfg.aniso ? potts_admm_step_t<S, true>(P, A, B, cfg.ac, cfg.plain, tmp, st)
                     : potts_admm_step_t<S, false>(P, A, B, cfg.ac, cfg.plain, tmp, st);
}

cudaError_t potts_step(int storage, const PottsProblem& P, const PottsStateV& a,
                       const PottsStateV& b, const StepConfig& cfg, float* tmp, cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return potts_step_s<float>(P, a, b, cfg, tmp, st);
        case CMF_F16: return potts_step_s<__half>(P, a, b, cfg, tmp, st);
        default: return potts_step_s<__nv_bfloat16>(P, a, b, cfg, tmp, st);
    }
}

template <typename S>
static cudaError_t potts_eval_s(const PottsProblem& P, const PottsStateV& sv, bool aniso, bool dr,
                                float tau, double* partials, cudaStream_t st,
                                const EvalTail& T) {
    const PottsState<S> s = sv.as<S>();
    const dim3 gr = pgrid(P.g, 8 * EVAL_ROWS), bl(32, 8);
    if (aniso) {
        if (dr) k_potts_eval<S, true, true><<<gr, bl, 0, st>>>(P, s, tau, partials, T);
        else k_potts_eval<S, true, false><<<gr, bl, 0, st>>>(P, s, tau, partials, T);
    } else {
        if (dr) k_potts_eval<S, false, true><<<gr, bl, 0, st>>>(P, s, tau, partials, T);
        else k_potts_eval<S, false, false><<<gr, bl, 0, st>>>(P, s, tau, partials, T);
    }
    return cudaGetLastError();
}

cudaError_t potts_eval(int storage, const PottsProblem& P, const PottsStateV& s, bool aniso,
                       bool dr, float tau, double* partials, cudaStream_t st, const EvalTail& T) {
    if (potts_strip_eligible(P.g, storage, P.C, P.alpha.plane, s, s))
        return potts_eval_strip(storage, P, s, aniso, dr, tau, partials, st, T);
    switch (storage) {
        case CMF_F32: return potts_eval_s<float>(P, s, aniso, dr, tau, partials, st, T);
        case CMF_F16: return potts_eval_s<__half>(P, s, aniso, dr, tau, partials, st, T);
        default: return potts_eval_s<__nv_bfloat16>(P, s, aniso, dr, tau, partials, st, T);
    }
}

}  // namespace cmf

// ---------------------------------------------------------------------------
// Batch kernels (see the binary ones): one block per tile of any Potts
// instance of a batch; dynamic shared memory sized for the largest L.
// ---------------------------------------------------------------------------
namespace cmf {

template <typename S, bool ANISO, int ROWS>
__global__ void __launch_bounds__(256)
    k_batch_potts_admm(const BatchDesc* desc, const int* tile_inst, int parity) {
    const BatchDesc* D = desc + tile_inst[blockIdx.x];
    if (!D->active) return;
    const int lt = blockIdx.x - D->tile_base;
    const PottsStateV a = parity ? D->pw : D->pu, b = parity ? D->pu : D->pw;
    potts_admm_tile<S, ANISO, ROWS>(D->pp, a.as<S>(), b.as<S>(), D->ak, lt % D->ntx,
                                    lt / D->ntx);
}

template <typename S, bool ANISO>
__global__ void __launch_bounds__(256)
    k_batch_potts_dr(const BatchDesc* desc, const int* tile_inst, int parity) {
    const BatchDesc* D = desc + tile_inst[blockIdx.x];
    if (!D->active) return;
    const int lt = blockIdx.x - D->tile_base;
    const PottsStateV a = parity ? D->pw : D->pu, b = parity ? D->pu : D->pw;
    potts_dr_tile<S, ANISO, 4, 1>(D->pp, a.as<S>(), b.as<S>(), D->dk, lt % D->ntx, lt / D->ntx);
}

template <typename S, bool ANISO, bool DR>
__global__ void __launch_bounds__(256)
    k_batch_potts_eval(const BatchDesc* desc, const int* tile_inst, float tau, double* partials) {
    const BatchDesc* D = desc + tile_inst[blockIdx.x];
    if (!D->active) return;
    const int lt = blockIdx.x - D->ev_tab;
    potts_eval_tile<S, ANISO, DR>(D->pp, D->pu.as<S>(), tau,
                                  partials + 3 * (size_t)(D->ev_base + lt), lt % D->ntx,
                                  lt / D->ntx);
}

template <typename S, bool ANISO, int ROWS>
static cudaError_t launch_batch_potts_admm(int maxL, const BatchDesc* desc, const int* tile_inst,
                                           int ntiles, int parity, cudaStream_t st) {
    const size_t dyn = (size_t)maxL * (8 * ROWS) * 32 * sizeof(float);
    auto kern = k_batch_potts_admm<S, ANISO, ROWS>;
    static std::atomic<long long> memo[kMaxDevices];  // limit set on each device
    {
        const cudaError_t e = raise_dyn_smem(memo, kern, dyn);
        if (e != cudaSuccess) return e;
    }
    kern<<<ntiles, dim3(32, 8), dyn, st>>>(desc, tile_inst, parity);
    return cudaGetLastError();
}

template <typename S, bool ANISO>
static cudaError_t batch_potts_step_t(bool dr, int rows, int maxL, const BatchDesc* desc,
                                      const int* tile_inst, int ntiles, int parity,
                                      cudaStream_t st) {
    if (dr) {
        k_batch_potts_dr<S, ANISO><<<ntiles, dim3(32, 8), 0, st>>>(desc, tile_inst, parity);
        return cudaGetLastError();
    }
    if (rows == 4) return launch_batch_potts_admm<S, ANISO, 4>(maxL, desc, tile_inst, ntiles, parity, st);
    if (rows == 2) return launch_batch_potts_admm<S, ANISO, 2>(maxL, desc, tile_inst, ntiles, parity, st);
    return launch_batch_potts_admm<S, ANISO, 1>(maxL, desc, tile_inst, ntiles, parity, st);
}

template <typename S>
static cudaError_t batch_potts_step_s(bool aniso, bool dr, int rows, int maxL,
                                      const BatchDesc* desc, const int* tile_inst, int ntiles,
                                      int parity, cudaStream_t st) {
    return aniso ? batch_potts_step_t<S, true>(dr, rows, maxL, desc, tile_inst, ntiles, parity, st)
                 : batch_potts_step_t<S, false>(dr, rows, maxL, desc, tile_inst, ntiles, parity, st);
}

cudaError_t batch_potts_step(int storage, bool aniso, bool dr, int sweeps, int rows, int maxL,
                             const BatchDesc* desc, const int* tile_inst, int ntiles,
                             int parity, cudaStream_t st) {
    if (dr && (sweeps != 1 || rows != 4)) return cudaErrorInvalidValue;
    switch (storage) {
        case CMF_F32: return batch_potts_step_s<float>(aniso, dr, rows, maxL, desc, tile_inst, ntiles, parity, st);
        case CMF_F16: return batch_potts_step_s<__half>(aniso, dr, rows, maxL, desc, tile_inst, ntiles, parity, st);
        default: return batch_potts_step_s<__nv_bfloat16>(aniso, dr, rows, maxL, desc, tile_inst, ntiles, parity, st);
    }
}

template <typename S>
static cudaError_t batch_potts_eval_s(bool aniso, bool dr, float tau, const BatchDesc* desc,
                                      const int* tile_inst, int ntiles, double* partials,
                                      cudaStream_t st) {
    const dim3 bl(32, 8);
    if (aniso) {
        if (dr) k_batch_potts_eval<S, true, true><<<ntiles, bl, 0, st>>>(desc, tile_inst, tau, partials);
        else k_batch_potts_eval<S, true, false><<<ntiles, bl, 0, st>>>(desc, tile_inst, tau, partials);
    } else {
        if (dr) k_batch_potts_eval<S, false, true><<<ntiles, bl, 0, st>>>(desc, tile_inst, tau, partials);
        else k_batch_potts_eval<S, false, false><<<ntiles, bl, 0, st>>>(desc, tile_inst, tau, partials);
    }
    return cudaGetLastError();
}

cudaError_t batch_potts_eval(int storage, bool aniso, bool dr, float tau,
                             const BatchDesc* desc, const int* tile_inst, int ntiles,
                             double* partials, cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return batch_potts_eval_s<float>(aniso, dr, tau, desc, tile_inst, ntiles, partials, st);
        case CMF_F16: return batch_potts_eval_s<__half>(aniso, dr, tau, desc, tile_inst, ntiles, partials, st);
        default: return batch_potts_eval_s<__nv_bfloat16>(aniso, dr, tau, desc, tile_inst, ntiles, partials, st);
    }
}

}  // namespace cmf
