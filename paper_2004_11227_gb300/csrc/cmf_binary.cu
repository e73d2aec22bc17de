// Binary continuous max-flow kernels (Eq. two-label-mf): cold start,
// rpADMMI / rpADMMII / pADMMI iterations (Eq. rpADMMI, Eq. rpADMMII),
// rPDRQ iterations (Eq. iteration:quadratic:seg) and the FP64-accumulated
// certificates (primal energy, max-flow value, conservation residual).
//
// Layout: every quantity is one row-major plane with row stride `pitch`.
// Thread blocks are 32 x 8; a block owns a 32-column x TY-row output tile.
//
// Fused forms (one kernel per iteration) read the state from one buffer set
// and write the next state to the other (ping-pong), because each output
// pixel needs neighbours' old values.  Plain forms launch one kernel per step
// of the method and update in place where the step allows it.
#include "cmf_kernels.cuh"

namespace cmf {

// ---------------------------------------------------------------------------
// Cold start: the alpha = 0 saddle point (u = 1 where C_t < C_s, q = 0,
// p_s = p_t = min(C_s, C_t)).  rPDRQ stores ybar = y - tau K u of that point:
// qbar = tau grad u, pbar_t = p_t - tau u, pbar_s = p_s + tau u.
// ---------------------------------------------------------------------------
template <typename S, bool DR>
__global__ void k_binary_init(BinProblem P, BinState<S> st, float tau) {
    const Grid G = P.g;
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int r = blockIdx.y * 8 + threadIdx.y;
    if (r >= G.H || c >= G.W) return;
    const size_t k = G.idx(r, c);
    const float cs = __ldg(P.Cs + k), ct = __ldg(P.Ct + k);
    const float u = ct < cs ? 1.0f : 0.0f;
    const float m = fminf(cs, ct);
    float qx = 0.f, qy = 0.f, ps = m, pt = m;
    if (DR) {
        if (c < G.W - 1) {
            const float ur = __ldg(P.Ct + k + 1) < __ldg(P.Cs + k + 1) ? 1.f : 0.f;
            qx = tau * (ur - u);
        }
        if (r < G.H - 1) {
            const size_t kd = k + G.pitch;
            const float ud = __ldg(P.Ct + kd) < __ldg(P.Cs + kd) ? 1.f : 0.f;
            qy = tau * (ud - u);
        }
        pt = m - tau * u;
        ps = m + tau * u;
    }
    st.u[k] = u;
    Store<S>::st(st.qx + k, qx);
    Store<S>::st(st.qy + k, qy);
    Store<S>::st(st.ps + k, ps);
    Store<S>::st(st.pt + k, pt);
}

// ---------------------------------------------------------------------------
// Fused ADMM iteration.  With g = div q^k + p_t^k - p_s^k - u^k / c the
// q-step of Eq. rpADMMII reads q^{k+1} = P_alpha(q^k + (1/a) grad g), since
// div^* = -grad.  The tile computes
//   phase 1: g on rows y0-1..y0+TY, cols x0-1..x0+32 (shared memory)
//   phase 2: q^{k+1} on rows y0-1..y0+TY-1, cols x0-1..x0+31
//   phase 3: d = div q^{k+1}, p^{k+1}, u^{k+1} on the tile.
// ---------------------------------------------------------------------------
template <typename S, bool ANISO, int ROWS>
__device__ __forceinline__ void binary_admm_tile(BinProblem P, BinState<S> s0, BinState<S> s1, AdmmCoef K, int bx_, int by_) {
    constexpr int TX = 32, TY = 8 * ROWS;
    constexpr int GX = TX + 2, GY = TY + 2;
    constexpr int QX = TX + 1, QY = TY + 1;
    __shared__ float g_s[GY][GX];
    __shared__ float qx_s[QY][QX];
    __shared__ float qy_s[QY][QX];
    using St = Store<S>;
    const Grid G = P.g;
    const int x0 = bx_ * TX, y0 = by_ * TY;
    const int tid = threadIdx.y * 32 + threadIdx.x;

    for (int i = tid; i < GX * GY; i += 256) {
        const int ly = i / GX, lx = i - ly * GX;
        const int r = y0 - 1 + ly, c = x0 - 1 + lx;
        float g = 0.f;
        if (r >= 0 && r < G.H && c >= 0 && c < G.W) {
            const size_t k = G.idx(r, c);
            float dv = 0.f;
            if (c < G.W - 1) dv += St::ld(s0.qx + k);
            if (c > 0) dv -= St::ld(s0.qx + k - 1);
            if (r < G.H - 1) dv += St::ld(s0.qy + k);
            if (r > 0) dv -= St::ld(s0.qy + k - G.pitch);
            g = dv + St::ld(s0.pt + k) - St::ld(s0.ps + k) - __ldg(s0.u + k) * K.inv_c;
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
            tx = St::ld(s0.qx + k) + (c < G.W - 1 ? (g_s[ly][lx + 1] - gc) * K.inv_a : 0.f);
            ty = St::ld(s0.qy + k) + (r < G.H - 1 ? (g_s[ly + 1][lx] - gc) * K.inv_a : 0.f);
            project_alpha<ANISO>(tx, ty, P.alpha.at(k));
            tx = St::rt(tx);
            ty = St::rt(ty);
            if (ly >= 1 && lx >= 1) {
                St::st(s1.qx + k, tx);
                St::st(s1.qy + k, ty);
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
        if (r < G.H && c < G.W) {
            const size_t k = G.idx(r, c);
            float d = 0.f;
            if (c < G.W - 1) d += qx_s[ly + 1][lx + 1];
            if (c > 0) d -= qx_s[ly + 1][lx];
            if (r < G.H - 1) d += qy_s[ly + 1][lx + 1];
            if (r > 0) d -= qy_s[ly][lx + 1];
            const float ps0 = St::ld(s0.ps + k), pt0 = St::ld(s0.pt + k);
            const float u0 = __ldg(s0.u + k);
            float ps1, pt1, u1;
            binary_pu<S>(K, g_s[ly + 1][lx + 1], d, ps0, pt0, u0, __ldg(P.Cs + k), __ldg(P.Ct + k),
                         ps1, pt1, u1);
            St::st(s1.ps + k, ps1);
            St::st(s1.pt + k, pt1);
            s1.u[k] = u1;
        }
    }
}

template <typename S, bool ANISO, int ROWS>
__global__ void __launch_bounds__(256)
    k_binary_admm_fused(BinProblem P, BinState<S> s0, BinState<S> s1, AdmmCoef K) {
    binary_admm_tile<S, ANISO, ROWS>(P, s0, s1, K, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Plain ADMM: one kernel per step, one thread per pixel.
// ---------------------------------------------------------------------------
#define PIXEL_PROLOGUE                                        \
    const Grid G = P.g;                                       \
    const int c = blockIdx.x * 32 + threadIdx.x;              \
    const int r = blockIdx.y * 8 + threadIdx.y;               \
    if (r >= G.H || c >= G.W) return;                         \
    const size_t k = G.idx(r, c);

template <typename S>
__device__ __forceinline__ float div_at(const Grid& G, const S* qx, const S* qy, int r, int c,
                                        size_t k) {
    using St = Store<S>;
    float v = 0.f;
    if (c < G.W - 1) v += St::ldw(qx + k);
    if (c > 0) v -= St::ldw(qx + k - 1);
    if (r < G.H - 1) v += St::ldw(qy + k);
    if (r > 0) v -= St::ldw(qy + k - G.pitch);
    return v;
}

// step a1: g = div q + p_t - p_s - u / c
template <typename S>
__global__ void k_binary_plain_g(BinProblem P, BinState<S> s, float* g, AdmmCoef K) {
    PIXEL_PROLOGUE
    using St = Store<S>;
    g[k] = div_at(G, s.qx, s.qy, r, c, k) + St::ldw(s.pt + k) - St::ldw(s.ps + k) -
           s.u[k] * K.inv_c;
}

// step a2: q = P_alpha(q + grad g / a), in place
template <typename S, bool ANISO>
__global__ void k_binary_plain_q(BinProblem P, BinState<S> s, const float* g, AdmmCoef K) {
    PIXEL_PROLOGUE
    using St = Store<S>;
    const float gc = g[k];
    float tx = St::ldw(s.qx + k) + (c < G.W - 1 ? (g[k + 1] - gc) * K.inv_a : 0.f);
    float ty = St::ldw(s.qy + k) + (r < G.H - 1 ? (g[k + G.pitch] - gc) * K.inv_a : 0.f);
    project_alpha<ANISO>(tx, ty, P.alpha.at(k));
    St::st(s.qx + k, tx);
    St::st(s.qy + k, ty);
}

// step a3: d = div q
template <typename S>
__global__ void k_binary_plain_div(BinProblem P, BinState<S> s, float* d) {
    PIXEL_PROLOGUE
    d[k] = div_at(G, s.qx, s.qy, r, c, k);
}

// steps a4 + a8: p and u updates, in place
template <typename S>
__global__ void k_binary_plain_pu(BinProblem P, BinState<S> s, const float* gbuf,
                                  const float* dbuf, AdmmCoef K) {
    PIXEL_PROLOGUE
    using St = Store<S>;
    const float d = dbuf[k];
    const float ps0 = St::ldw(s.ps + k), pt0 = St::ldw(s.pt + k), u0 = s.u[k];
    float ps1, pt1, u1;
    binary_pu<S>(K, gbuf[k], d, ps0, pt0, u0, __ldg(P.Cs + k), __ldg(P.Ct + k), ps1, pt1, u1);
    St::st(s.ps + k, ps1);
    St::st(s.pt + k, pt1);
    s.u[k] = u1;
}

// ---------------------------------------------------------------------------
// rPDRQ (Eq. iteration:quadratic:seg).  State (u, qbar, pbar_s, pbar_t).
//   b = -sigma (div qbar + pbar_t - pbar_s)
//   u <- sRBGS sweep(s) on sigma tau (2 I - Lap) u = b: red, (black, red) x s
//   q = qbar - tau grad u, p_t = pbar_t + tau u, p_s = pbar_s - tau u
//   qbar += rho (P_alpha(2q - qbar) - q)
//   pbar_t += rho (min(2 p_t - pbar_t, C_t) - p_t)
//   pbar_s += rho (min(2 p_s - pbar_s + tau, C_s) - p_s)
// ---------------------------------------------------------------------------
// Fused: the tile's u after h = 2 sweeps + 1 half-sweeps is needed on rows
// y0..y0+TY and cols x0..x0+32 (one extra for grad u).  Half-sweep s updates
// its colour on that region grown by h-1-s, so u^k is staged on the region
// grown by h and b on the region grown by h-1.
template <typename S, bool ANISO, int ROWS, int SW>
__device__ __forceinline__ void binary_dr_tile(BinProblem P, BinState<S> s0, BinState<S> s1, DrCoef D, int bx_, int by_) {
    constexpr int TX = 32, TY = 8 * ROWS;
    constexpr int NH = 2 * SW + 1;
    constexpr int UX = TX + 1 + 2 * NH, UY = TY + 1 + 2 * NH;
    constexpr int BX = UX - 2, BY = UY - 2;
    __shared__ float u_s[UY][UX];
    __shared__ float b_s[BY][BX];
    using St = Store<S>;
    const Grid G = P.g;
    const int x0 = bx_ * TX, y0 = by_ * TY;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int ux0 = x0 - NH, uy0 = y0 - NH;  // grid coords of u_s[0][0]

    for (int i = tid; i < UX * UY; i += 256) {
        const int ly = i / UX, lx = i - ly * UX;
        const int r = uy0 + ly, c = ux0 + lx;
        float v = 0.f;
        if (r >= 0 && r < G.H && c >= 0 && c < G.W) v = __ldg(s0.u + G.idx(r, c));
        u_s[ly][lx] = v;
    }
    for (int i = tid; i < BX * BY; i += 256) {
        const int ly = i / BX, lx = i - ly * BX;
        const int r = uy0 + 1 + ly, c = ux0 + 1 + lx;
        float b = 0.f;
        if (r >= 0 && r < G.H && c >= 0 && c < G.W) {
            const size_t k = G.idx(r, c);
            float dv = 0.f;
            if (c < G.W - 1) dv += St::ld(s0.qx + k);
            if (c > 0) dv -= St::ld(s0.qx + k - 1);
            if (r < G.H - 1) dv += St::ld(s0.qy + k);
            if (r > 0) dv -= St::ld(s0.qy + k - G.pitch);
            b = -D.sigma * (dv + St::ld(s0.pt + k) - St::ld(s0.ps + k));
        }
        b_s[ly][lx] = b;
    }
    __syncthreads();

#pragma unroll 1
    for (int s = 0; s < NH; ++s) {
        const int colour = s & 1;  // red (i+j even) first
        const int grow = NH - 1 - s;
        // region in u_s coordinates: [NH - grow, NH + TY + grow] (inclusive)
        const int lo = NH - grow;
        const int ny = TY + 1 + 2 * grow, nx = TX + 1 + 2 * grow;
        for (int i = tid; i < nx * ny; i += 256) {
            const int ly = lo + i / nx, lx = lo + i % nx;
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
            float oqx, oqy, ops, opt;
            binary_dr_flows<S, ANISO>(D, uc, gx, gy, St::ld(s0.qx + k), St::ld(s0.qy + k),
                                      St::ld(s0.ps + k), St::ld(s0.pt + k), P.alpha.at(k),
                                      __ldg(P.Cs + k), __ldg(P.Ct + k), oqx, oqy, ops, opt);
            s1.u[k] = uc;
            St::st(s1.qx + k, oqx);
            St::st(s1.qy + k, oqy);
            St::st(s1.ps + k, ops);
            St::st(s1.pt + k, opt);
        }
    }
}

template <typename S, bool ANISO, int ROWS, int SW>
__global__ void __launch_bounds__(256)
    k_binary_dr_fused(BinProblem P, BinState<S> s0, BinState<S> s1, DrCoef D) {
    binary_dr_tile<S, ANISO, ROWS, SW>(P, s0, s1, D, blockIdx.x, blockIdx.y);
}

// Plain rPDRQ: b, then one kernel per red/black half-sweep (in place: a
// half-sweep reads only the other colour), then the flow reflections.
template <typename S>
__global__ void k_binary_plain_dr_b(BinProblem P, BinState<S> s, float* b, DrCoef D) {
    PIXEL_PROLOGUE
    using St = Store<S>;
    b[k] = -D.sigma * (div_at(G, s.qx, s.qy, r, c, k) + St::ldw(s.pt + k) - St::ldw(s.ps + k));
}

__global__ void k_plain_halfsweep(Grid G, float* u, const float* b, float inv_st, float kappa,
                                  int colour) {
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int r = blockIdx.y * 8 + threadIdx.y;
    if (r >= G.H || c >= G.W || ((r + c) & 1) != colour) return;
    const size_t k = G.idx(r, c);
    float sum = 0.f;
    int nnb = 0;
    if (c > 0) { sum += u[k - 1]; ++nnb; }
    if (c < G.W - 1) { sum += u[k + 1]; ++nnb; }
    if (r > 0) { sum += u[k - G.pitch]; ++nnb; }
    if (r < G.H - 1) { sum += u[k + G.pitch]; ++nnb; }
    u[k] = (b[k] * inv_st + sum) / (kappa + (float)nnb);
}

// Red, then (black, red) x sweeps, one launch per half-sweep.
cudaError_t halfsweeps(const Grid& G, float* u, const float* b, const DrCoef& D,
                       cudaStream_t st) {
    const dim3 gr((G.W + 31) / 32, (G.H + 7) / 8), bl(32, 8);
    k_plain_halfsweep<<<gr, bl, 0, st>>>(G, u, b, D.inv_st, D.kappa, 0);
    for (int s = 0; s < D.sweeps; ++s) {
        k_plain_halfsweep<<<gr, bl, 0, st>>>(G, u, b, D.inv_st, D.kappa, 1);
        k_plain_halfsweep<<<gr, bl, 0, st>>>(G, u, b, D.inv_st, D.kappa, 0);
    }
    return cudaGetLastError();
}

template <typename S, bool ANISO>
__global__ void k_binary_plain_dr_flows(BinProblem P, BinState<S> s, DrCoef D) {
    PIXEL_PROLOGUE
    using St = Store<S>;
    const float uc = s.u[k];
    const float gx = c < G.W - 1 ? s.u[k + 1] - uc : 0.f;
    const float gy = r < G.H - 1 ? s.u[k + G.pitch] - uc : 0.f;
    float oqx, oqy, ops, opt;
    binary_dr_flows<S, ANISO>(D, uc, gx, gy, St::ldw(s.qx + k), St::ldw(s.qy + k),
                              St::ldw(s.ps + k), St::ldw(s.pt + k), P.alpha.at(k),
                              __ldg(P.Cs + k), __ldg(P.Ct + k), oqx, oqy, ops, opt);
    St::st(s.qx + k, oqx);
    St::st(s.qy + k, oqy);
    St::st(s.ps + k, ops);
    St::st(s.pt + k, opt);
}

// ---------------------------------------------------------------------------
// Certificates (FP64 accumulation).  A block owns a 32 x TY tile (TY = 8 x
// EVAL_ROWS): u is staged on the tile grown by one row / column on each side,
// the flows y and their projections P_alpha(y) on the tile grown by one on
// the low side, all in shared memory; per-pixel terms are float32, sums are
// float64; one partial triple (E, D, res^2) per block, reduced in a fixed
// order by k_reduce_partials.  For rPDRQ y = ybar + tau K u.
// ---------------------------------------------------------------------------
template <typename S, bool ANISO, bool DR>
__device__ __forceinline__ void binary_eval_tile(BinProblem P, BinState<S> s, float tau, double* out3, int bx_, int by_) {
    constexpr int TX = 32, TY = 8 * EVAL_ROWS;
    __shared__ float u_s[TY + 2][TX + 2];   // grid (y0-1+i, x0-1+j)
    __shared__ float fx_s[TY + 1][TX + 1];  // grid (y0-1+i, x0-1+j)
    __shared__ float fy_s[TY + 1][TX + 1];
    __shared__ float px_s[TY + 1][TX + 1];
    __shared__ float py_s[TY + 1][TX + 1];
    using St = Store<S>;
    const Grid G = P.g;
    const int x0 = bx_ * TX, y0 = by_ * TY;
    const int tid = threadIdx.y * 32 + threadIdx.x;

    for (int i = tid; i < (TY + 2) * (TX + 2); i += 256) {
        const int a = i / (TX + 2), b = i - a * (TX + 2);
        const int r = y0 - 1 + a, c = x0 - 1 + b;
        u_s[a][b] = (r >= 0 && r < G.H && c >= 0 && c < G.W) ? s.u[G.idx(r, c)] : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < (TY + 1) * (TX + 1); i += 256) {
        const int a = i / (TX + 1), b = i - a * (TX + 1);
        const int r = y0 - 1 + a, c = x0 - 1 + b;
        float fx = 0.f, fy = 0.f, px = 0.f, py = 0.f;
        if (r >= 0 && r < G.H && c >= 0 && c < G.W) {
            const size_t k = G.idx(r, c);
            fx = St::ldw(s.qx + k);
            fy = St::ldw(s.qy + k);
            if (DR) {
                const float uc = u_s[a][b];
                if (c < G.W - 1) fx -= tau * (u_s[a][b + 1] - uc);
                if (r < G.H - 1) fy -= tau * (u_s[a + 1][b] - uc);
            }
            px = fx;
            py = fy;
            project_alpha<ANISO>(px, py, P.alpha.at(k));
        }
        fx_s[a][b] = fx;
        fy_s[a][b] = fy;
        px_s[a][b] = px;
        py_s[a][b] = py;
    }
    __syncthreads();

    DF accE = {0.f, 0.f}, accD = {0.f, 0.f}, accR = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < EVAL_ROWS; ++j) {
        const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
        const int r = y0 + ly, c = x0 + lx;
        if (r >= G.H || c >= G.W) continue;
        const size_t k = G.idx(r, c);
        const float cs = __ldg(P.Cs + k), ct = __ldg(P.Ct + k);
        const float al = P.alpha.at(k);
        // primal energy at ub = clip(u, 0, 1)
        const float uc = u_s[ly + 1][lx + 1];
        const float ub = fminf(fmaxf(uc, 0.f), 1.f);
        const float gx = c < G.W - 1 ? fminf(fmaxf(u_s[ly + 1][lx + 2], 0.f), 1.f) - ub : 0.f;
        const float gy = r < G.H - 1 ? fminf(fmaxf(u_s[ly + 2][lx + 1], 0.f), 1.f) - ub : 0.f;
        const float tv = ANISO ? fabsf(gx) + fabsf(gy) : sqrtf(gx * gx + gy * gy);
        df_add(accE, (1.f - ub) * cs + ub * ct + al * tv);
        // conservation residual of y, and the max-flow value of P_alpha(y);
        // out-of-grid neighbours of the tile hold 0
        float ps = St::ldw(s.ps + k), pt = St::ldw(s.pt + k);
        if (DR) {
            pt += tau * uc;
            ps -= tau * uc;
        }
        const float dv = (c < G.W - 1 ? fx_s[ly + 1][lx + 1] : 0.f) - fx_s[ly + 1][lx] +
                         (r < G.H - 1 ? fy_s[ly + 1][lx + 1] : 0.f) - fy_s[ly][lx + 1];
        const float rr = dv - ps + pt;
        df_add(accR, rr * rr);
        const float dp = (c < G.W - 1 ? px_s[ly + 1][lx + 1] : 0.f) - px_s[ly + 1][lx] +
                         (r < G.H - 1 ? py_s[ly + 1][lx + 1] : 0.f) - py_s[ly][lx + 1];
        df_add(accD, fminf(cs, ct + dp));
    }
    block_reduce3_store_df(accE, accD, accR, out3);
}

template <typename S, bool ANISO, bool DR>
__global__ void __launch_bounds__(256)
    k_binary_eval(BinProblem P, BinState<S> s, float tau, double* partials, EvalTail T) {
    binary_eval_tile<S, ANISO, DR>(P, s, tau, partials + 3 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x), blockIdx.x, blockIdx.y);
    eval_tail(T, partials, gridDim.x * gridDim.y);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static inline dim3 grid_for(const Grid& G, int rows_per_block) {
    return dim3((G.W + 31) / 32, (G.H + rows_per_block - 1) / rows_per_block);
}

template <typename S>
static cudaError_t binary_init_t(const BinProblem& P, const BinState<S>& s, bool dr, float tau,
                                 cudaStream_t st) {
    if (dr)
        k_binary_init<S, true><<<grid_for(P.g, 8), dim3(32, 8), 0, st>>>(P, s, tau);
    else
        k_binary_init<S, false><<<grid_for(P.g, 8), dim3(32, 8), 0, st>>>(P, s, tau);
    return cudaGetLastError();
}

cudaError_t binary_init(int storage, const BinProblem& P, const BinStateV& s, bool dr, float tau,
                        cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return binary_init_t<float>(P, s.as<float>(), dr, tau, st);
        case CMF_F16: return binary_init_t<__half>(P, s.as<__half>(), dr, tau, st);
        default: return binary_init_t<__nv_bfloat16>(P, s.as<__nv_bfloat16>(), dr, tau, st);
    }
}

template <typename S, bool ANISO>
static cudaError_t binary_admm_step_t(const BinProblem& P, const BinState<S>& a,
                                      const BinState<S>& b, const AdmmCoef& K, bool plain,
                                      float* tmp, cudaStream_t st) {
    if (!plain) {
        constexpr int ROWS = 4;
        k_binary_admm_fused<S, ANISO, ROWS>
            <<<grid_for(P.g, 8 * ROWS), dim3(32, 8), 0, st>>>(P, a, b, K);
        return cudaGetLastError();
    }
    const dim3 gr = grid_for(P.g, 8), bl(32, 8);
    k_binary_plain_g<S><<<gr, bl, 0, st>>>(P, a, tmp, K);
    k_binary_plain_q<S, ANISO><<<gr, bl, 0, st>>>(P, a, tmp, K);
    k_binary_plain_div<S><<<gr, bl, 0, st>>>(P, a, tmp + P.g.plane);
    k_binary_plain_pu<S><<<gr, bl, 0, st>>>(P, a, tmp, tmp + P.g.plane, K);
    return cudaGetLastError();
}

template <typename S, bool ANISO>
static cudaError_t binary_dr_step_t(const BinProblem& P, const BinState<S>& a,
                                    const BinState<S>& b, const DrCoef& D, bool plain,
                                    float* tmp, cudaStream_t st) {
    if (!plain) {
        constexpr int ROWS = 4;
        const dim3 gr = grid_for(P.g, 8 * ROWS), bl(32, 8);
        switch (D.sweeps) {
            case 1: k_binary_dr_fused<S, ANISO, ROWS, 1><<<gr, bl, 0, st>>>(P, a, b, D); break;
            case 2: k_binary_dr_fused<S, ANISO, ROWS, 2><<<gr, bl, 0, st>>>(P, a, b, D); break;
            case 3: k_binary_dr_fused<S, ANISO, ROWS, 3><<<gr, bl, 0, st>>>(P, a, b, D); break;
            default: k_binary_dr_fused<S, ANISO, ROWS, 4><<<gr, bl, 0, st>>>(P, a, b, D); break;
        }
        return cudaGetLastError();
    }
    const dim3 gr = grid_for(P.g, 8), bl(32, 8);
    k_binary_plain_dr_b<S><<<gr, bl, 0, st>>>(P, a, tmp, D);
    cudaError_t e = halfsweeps(P.g, a.u, tmp, D, st);
    if (e != cudaSuccess) return e;
    k_binary_plain_dr_flows<S, ANISO><<<gr, bl, 0, st>>>(P, a, D);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t binary_step_s(const BinProblem& P, const BinStateV& a, const BinStateV& b,
                                 const StepConfig& cfg, float* tmp, cudaStream_t st) {
    const BinState<S> A = a.as<S>(), B = b.as<S>();
    if (cfg.dr) {
        return cfg.aniso ? binary_dr_step_t<S, true>(P, A, B, cfg.dc, cfg.plain, tmp, st)
                         : binary_dr_step_t<S, false>(P, A, B, cfg.dc, cfg.plain, tmp, st);
    }
    return cfg.aniso ? binary_admm_step_t<S, true>(P, A, B, cfg.ac, cfg.plain, tmp, st)
                     : binary_admm_step_t<S, false>(P, A, B, cfg.ac, cfg.plain, tmp, st);
}

cudaError_t binary_step(int storage, const BinProblem& P, const BinStateV& a, const BinStateV& b,
                        const StepConfig& cfg, float* tmp, cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return binary_step_s<float>(P, a, b, cfg, tmp, st);
        case CMF_F16: return binary_step_s<__half>(P, a, b, cfg, tmp, st);
        default: return binary_step_s<__nv_bfloat16>(P, a, b, cfg, tmp, st);
    }
}

template <typename S>
static cudaError_t binary_eval_s(const BinProblem& P, const BinStateV& sv, bool aniso, bool dr,
                                 float tau, double* partials, cudaStream_t st,
                                 const EvalTail& T) {
    const BinState<S> s = sv.as<S>();
    const dim3 gr = grid_for(P.g, 8 * EVAL_ROWS), bl(32, 8);
    if (aniso) {
        if (dr) k_binary_eval<S, true, true><<<gr, bl, 0, st>>>(P, s, tau, partials, T);
        else k_binary_eval<S, true, false><<<gr, bl, 0, st>>>(P, s, tau, partials, T);
    } else {
        if (dr) k_binary_eval<S, false, true><<<gr, bl, 0, st>>>(P, s, tau, partials, T);
        else k_binary_eval<S, false, false><<<gr, bl, 0, st>>>(P, s, tau, partials, T);
    }
    return cudaGetLastError();
}

cudaError_t binary_eval(int storage, const BinProblem& P, const BinStateV& s, bool aniso, bool dr,
                        float tau, double* partials, cudaStream_t st, const EvalTail& T) {
    const float* al = P.alpha.plane;
    if (binary_strip_eligible(P.g, storage, P.Cs, P.Ct, al, s, s))
        return binary_eval_strip(storage, P, s, aniso, dr, tau, partials, st, T);
    switch (storage) {
        case CMF_F32: return binary_eval_s<float>(P, s, aniso, dr, tau, partials, st, T);
        case CMF_F16: return binary_eval_s<__half>(P, s, aniso, dr, tau, partials, st, T);
        default: return binary_eval_s<__nv_bfloat16>(P, s, aniso, dr, tau, partials, st, T);
    }
}

int eval_blocks(int H, int W) { return ((W + 31) / 32) * ((H + 8 * EVAL_ROWS - 1) / (8 * EVAL_ROWS)); }

}  // namespace cmf

// ---------------------------------------------------------------------------
// Batch kernels: one block per tile of any binary instance of a batch; the
// block finds its instance through the tile table and returns at once when
// that instance has converged.
// ---------------------------------------------------------------------------
namespace cmf {

template <typename S, bool ANISO>
__global__ void __launch_bounds__(256)
    k_batch_binary_admm(const BatchDesc* desc, const int* tile_inst, int parity) {
    const BatchDesc* D = desc + tile_inst[blockIdx.x];
    if (!D->active) return;
    const int lt = blockIdx.x - D->tile_base;
    const BinStateV a = parity ? D->bw : D->bu, b = parity ? D->bu : D->bw;
    binary_admm_tile<S, ANISO, 4>(D->bp, a.as<S>(), b.as<S>(), D->ak, lt % D->ntx, lt / D->ntx);
}

template <typename S, bool ANISO>
__global__ void __launch_bounds__(256)
    k_batch_binary_dr(const BatchDesc* desc, const int* tile_inst, int parity) {
    const BatchDesc* D = desc + tile_inst[blockIdx.x];
    if (!D->active) return;
    const int lt = blockIdx.x - D->tile_base;
    const BinStateV a = parity ? D->bw : D->bu, b = parity ? D->bu : D->bw;
    binary_dr_tile<S, ANISO, 4, 1>(D->bp, a.as<S>(), b.as<S>(), D->dk, lt % D->ntx, lt / D->ntx);
}

template <typename S, bool ANISO, bool DR>
__global__ void __launch_bounds__(256)
    k_batch_binary_eval(const BatchDesc* desc, const int* tile_inst, float tau,
                        double* partials) {
    const BatchDesc* D = desc + tile_inst[blockIdx.x];
    if (!D->active) return;
    const int lt = blockIdx.x - D->ev_tab;
    binary_eval_tile<S, ANISO, DR>(D->bp, D->bu.as<S>(), tau,
                                   partials + 3 * (size_t)(D->ev_base + lt), lt % D->ntx,
                                   lt / D->ntx);
}

template <typename S>
static cudaError_t batch_binary_step_s(bool aniso, bool dr, const BatchDesc* desc,
                                       const int* tile_inst, int ntiles, int parity,
                                       cudaStream_t st) {
    const dim3 bl(32, 8);
    if (dr) {
        if (aniso) k_batch_binary_dr<S, true><<<ntiles, bl, 0, st>>>(desc, tile_inst, parity);
        else k_batch_binary_dr<S, false><<<ntiles, bl, 0, st>>>(desc, tile_inst, parity);
    } else {
        if (aniso) k_batch_binary_admm<S, true><<<ntiles, bl, 0, st>>>(desc, tile_inst, parity);
        else k_batch_binary_admm<S, false><<<ntiles, bl, 0, st>>>(desc, tile_inst, parity);
    }
    return cudaGetLastError();
}

cudaError_t batch_binary_step(int storage, bool aniso, bool dr, int sweeps,
                              const BatchDesc* desc, const int* tile_inst, int ntiles,
                              int parity, cudaStream_t st) {
    if (dr && sweeps != 1) return cudaErrorInvalidValue;
    switch (storage) {
        case CMF_F32: return batch_binary_step_s<float>(aniso, dr, desc, tile_inst, ntiles, parity, st);
        case CMF_F16: return batch_binary_step_s<__half>(aniso, dr, desc, tile_inst, ntiles, parity, st);
        default: return batch_binary_step_s<__nv_bfloat16>(aniso, dr, desc, tile_inst, ntiles, parity, st);
    }
}

template <typename S>
static cudaError_t batch_binary_eval_s(bool aniso, bool dr, float tau, const BatchDesc* desc,
                                       const int* tile_inst, int ntiles, double* partials,
                                       cudaStream_t st) {
    const dim3 bl(32, 8);
    if (aniso) {
        if (dr) k_batch_binary_eval<S, true, true><<<ntiles, bl, 0, st>>>(desc, tile_inst, tau, partials);
        else k_batch_binary_eval<S, true, false><<<ntiles, bl, 0, st>>>(desc, tile_inst, tau, partials);
    } else {
        if (dr) k_batch_binary_eval<S, false, true><<<ntiles, bl, 0, st>>>(desc, tile_inst, tau, partials);
        else k_batch_binary_eval<S, false, false><<<ntiles, bl, 0, st>>>(desc, tile_inst, tau, partials);
    }
    return cudaGetLastError();
}

cudaError_t batch_binary_eval(int storage, bool aniso, bool dr, float tau,
                              const BatchDesc* desc, const int* tile_inst, int ntiles,
                              double* partials, cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return batch_binary_eval_s<float>(aniso, dr, tau, desc, tile_inst, ntiles, partials, st);
        case CMF_F16: return batch_binary_eval_s<__half>(aniso, dr, tau, desc, tile_inst, ntiles, partials, st);
        default: return batch_binary_eval_s<__nv_bfloat16>(aniso, dr, tau, desc, tile_inst, ntiles, partials, st);
    }
}

}  // namespace cmf
