// Potts ADMM iteration with TMA-staged label planes (Eq. multi:fg:4 and the
// Eckstein-Bertsekas Potts equations after Thm 2, general L).
//
// A block owns a 32 x TY output tile and walks the L labels.  For each label
// the four state planes it reads with a halo (q_x, q_y, p_i, u_i) arrive as
// TMA boxes in a shared-memory stage; two stages alternate, so label l+2 is
// in flight while label l is computed.  p_s arrives once.  Everything the
// iteration reads with a halo then comes from shared memory; only the costs,
// alpha and the outputs touch global memory directly.
//
// Staged box of a field: rows y0-2 .. y0+TY, columns x0-XO .. x0-XO+BX-1
// (XO = 4 for 4-byte elements and 8 for 2-byte ones, so the box starts on a
// 16-byte boundary); elements outside the grid read as zero.
#include "cmf_kernels.cuh"
#include "cmf_tma.cuh"

namespace cmf {

namespace {

constexpr int align128(int b) { return (b + 127) / 128 * 128; }

template <typename S, int TY>
struct PottsTmaLayout {
    static constexpr int BY = TY + 3;
    static constexpr int XO = sizeof(S) == 4 ? 4 : 8;
    static constexpr int BXS = sizeof(S) == 4 ? 40 : 48;
    static constexpr int XU = 4, BXU = 40;
    static constexpr int FS = align128(BY * BXS * (int)sizeof(S));
    static constexpr int FU = align128(BY * BXU * 4);
    static constexpr int STAGE = 3 * FS + FU;
    static constexpr uint32_t TX_BYTES = 3u * BY * BXS * sizeof(S) + (uint32_t)BY * BXU * 4u;
    static constexpr uint32_t PS_BYTES = (uint32_t)BY * BXS * sizeof(S);
    // + 128: the kernel rounds the dynamic shared-memory base up to 128 bytes
    static size_t dyn_bytes(int L) { return 2 * STAGE + FS + (size_t)L * TY * 32 * 4 + 128; }
};

template <typename S>
__device__ __forceinline__ float sload(const S* p) {
    return Store<S>::ldw(p);
}

}  // namespace

template <typename S, bool ANISO, int TY>
__global__ void __launch_bounds__(256)
    k_potts_admm_tma(PottsProblem P, PottsState<S> s1, AdmmCoef K,
                     const __grid_constant__ CUtensorMap mqx,
                     const __grid_constant__ CUtensorMap mqy,
                     const __grid_constant__ CUtensorMap mp,
                     const __grid_constant__ CUtensorMap mu,
                     const __grid_constant__ CUtensorMap mps, int* err) {
    using Lay = PottsTmaLayout<S, TY>;
    using St = Store<S>;
    constexpr int TX = 32, ROWS = TY / 8;
    constexpr int BXS = Lay::BXS, BXU = Lay::BXU, XO = Lay::XO, XU = Lay::XU;
    __shared__ __align__(8) uint64_t bar[3];
    __shared__ float g_s[TY + 2][TX + 2];
    __shared__ float qnx[TY + 1][TX + 1];
    __shared__ float qny[TY + 1][TX + 1];
    extern __shared__ __align__(128) unsigned char dsm_raw[];
    unsigned char* dsm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(dsm_raw) + 127) & ~static_cast<uintptr_t>(127));
    unsigned char* stage[2] = {dsm, dsm + Lay::STAGE};
    S* ps_s = reinterpret_cast<S*>(dsm + 2 * Lay::STAGE);
    float* v_s = reinterpret_cast<float*>(dsm + 2 * Lay::STAGE + Lay::FS);

    const Grid G = P.g;
    const int L = P.L;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

    auto issue = [&](int l, int s) {
        unsigned char* d = stage[s];
        mbar_arrive_expect_tx(&bar[s], Lay::TX_BYTES);
        tma_load_3d(d, &mqx, &bar[s], x0 - XO, y0 - 2, l);
        tma_load_3d(d + Lay::FS, &mqy, &bar[s], x0 - XO, y0 - 2, l);
        tma_load_3d(d + 2 * Lay::FS, &mp, &bar[s], x0 - XO, y0 - 2, l);
        tma_load_3d(d + 3 * Lay::FS, &mu, &bar[s], x0 - XU, y0 - 2, l);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar[2], Lay::PS_BYTES);
        tma_load_3d(ps_s, &mps, &bar[2], x0 - XO, y0 - 2, 0);
        issue(0, 0);
        if (L > 1) issue(1, 1);
    }
    bool ok = mbar_wait_bounded(&bar[2], 0, kWaitLimitCycles);

    float accd[ROWS], accp[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) accd[j] = accp[j] = 0.f;

#pragma unroll 1
    for (int l = 0; l < L; ++l) {
        const int s = l & 1;
        const S* sqx = reinterpret_cast<const S*>(stage[s]);
        const S* sqy = reinterpret_cast<const S*>(stage[s] + Lay::FS);
        const S* sp = reinterpret_cast<const S*>(stage[s] + 2 * Lay::FS);
        const float* su = reinterpret_cast<const float*>(stage[s] + 3 * Lay::FS);
        ok = ok && mbar_wait_bounded(&bar[s], (l >> 1) & 1, kWaitLimitCycles);
        if (__syncthreads_or(!ok)) {
            // a TMA stage never arrived: flag it, give in-flight copies a
            // bounded chance to land in this block's shared memory, return
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait_bounded(&bar[0], (l >> 1) & 1, kWaitLimitCycles);
                if (L > 1) mbar_wait_bounded(&bar[1], (l >> 1) & 1, kWaitLimitCycles);
            }
            return;
        }
        const size_t lo = (size_t)l * G.plane;

        // g_l on rows y0-1..y0+TY, cols x0-1..x0+TX
        for (int i = tid; i < (TY + 2) * (TX + 2); i += 256) {
            const int gy = i / (TX + 2), gx = i - gy * (TX + 2);
            const int r = y0 - 1 + gy, c = x0 - 1 + gx;
            const int sy = gy + 1, sx = gx - 1 + XO, su_x = gx - 1 + XU;
            // neighbours outside the grid were zero-filled by the TMA unit
            float dv = 0.f;
            if (c < G.W - 1) dv += sload(sqx + sy * BXS + sx);
            dv -= sload(sqx + sy * BXS + sx - 1);
            if (r < G.H - 1) dv += sload(sqy + sy * BXS + sx);
            dv -= sload(sqy + (sy - 1) * BXS + sx);
            g_s[gy][gx] = dv + sload(sp + sy * BXS + sx) - sload(ps_s + sy * BXS + sx) -
                          su[sy * BXU + su_x] * K.inv_c;
        }
        __syncthreads();

        // q_l^{k+1} on rows y0-1..y0+TY-1, cols x0-1..x0+TX-1
        for (int i = tid; i < (TY + 1) * (TX + 1); i += 256) {
            const int qy_ = i / (TX + 1), qx_ = i - qy_ * (TX + 1);
            const int r = y0 - 1 + qy_, c = x0 - 1 + qx_;
            float tx = 0.f, ty = 0.f;
            if (r >= 0 && r < G.H && c >= 0 && c < G.W) {
                const int sy = qy_ + 1, sx = qx_ - 1 + XO;
                const size_t k = G.idx(r, c);
                const float gc = g_s[qy_][qx_];
                tx = sload(sqx + sy * BXS + sx) +
                     (c < G.W - 1 ? (g_s[qy_][qx_ + 1] - gc) * K.inv_a : 0.f);
                ty = sload(sqy + sy * BXS + sx) +
                     (r < G.H - 1 ? (g_s[qy_ + 1][qx_] - gc) * K.inv_a : 0.f);
                project_alpha<ANISO>(tx, ty, P.alpha.at(k));
                tx = St::rt(tx);
                ty = St::rt(ty);
                if (qy_ >= 1 && qx_ >= 1) {
                    St::st(s1.qx + lo + k, tx);
                    St::st(s1.qy + lo + k, ty);
                }
            }
            qnx[qy_][qx_] = tx;
            qny[qy_][qx_] = ty;
        }
        __syncthreads();

        // d_l, p_l^{k+1}, the p_s terms and v_l on the tile
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
            const int r = y0 + ly, c = x0 + lx;
            float v = 0.f;
            if (r < G.H && c < G.W) {
                const size_t k = G.idx(r, c);
                float d = 0.f;  // out-of-grid neighbours of the q tile hold 0
                if (c < G.W - 1) d += qnx[ly + 1][lx + 1];
                d -= qnx[ly + 1][lx];
                if (r < G.H - 1) d += qny[ly + 1][lx + 1];
                d -= qny[ly][lx + 1];
                const int sy = ly + 2;
                const float ps0 = sload(ps_s + sy * BXS + lx + XO);
                const float p0 = sload(sp + sy * BXS + lx + XO);
                const float u0 = su[sy * BXU + lx + XU];
                float p1 = fminf(p0 - (K.rho_p * (p0 - ps0) - u0 * K.inv_c + K.rho_p * d) * K.inv_a1,
                                 __ldg(P.C + lo + k));
                p1 = St::rt(p1);
                St::st(s1.p + lo + k, p1);
                accd[j] += K.rho_p * d;
                accp[j] += K.rho_p * (p0 - ps0) - u0 * K.inv_c;
                v = u0 - K.cu * (p1 - K.omr * (p0 - ps0) + K.rho_p * d);
            }
            v_s[(l * TY + ly) * TX + lx] = v;
        }
        __syncthreads();
        if (tid == 0 && l + 2 < L) {
            fence_proxy_async_smem();
            issue(l + 2, s);
        }
    }

    float ps1[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
        const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
        const int r = y0 + ly, c = x0 + lx;
        ps1[j] = 0.f;
        if (r < G.H && c < G.W) {
            const float ps0 = sload(ps_s + (ly + 2) * BXS + lx + XO);
            ps1[j] = St::rt(ps0 + (accd[j] + accp[j] + K.inv_c) * K.inv_a2);
            St::st(s1.ps + G.idx(r, c), ps1[j]);
        }
    }
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
            const int r = y0 + ly, c = x0 + lx;
            if (r < G.H && c < G.W)
                s1.u[(size_t)l * G.plane + G.idx(r, c)] =
                    v_s[(l * TY + ly) * TX + lx] + K.cu * ps1[j];
        }
    }
}

// Shared memory one block of the TMA kernel needs (static + dynamic).
static size_t tma_smem_bytes(int storage, int L, int ty) {
    const size_t stat = (size_t)(ty + 2) * 34 * 4 + 2 * (size_t)(ty + 1) * 33 * 4 + 64;
    size_t dyn;
    if (storage == CMF_F32)
        dyn = ty == 32 ? PottsTmaLayout<float, 32>::dyn_bytes(L)
                       : PottsTmaLayout<float, 16>::dyn_bytes(L);
    else
        dyn = ty == 32 ? PottsTmaLayout<__half, 32>::dyn_bytes(L)
                       : PottsTmaLayout<__half, 16>::dyn_bytes(L);
    return stat + dyn;
}

bool potts_tma_fits(int storage, int L, int ty) {
    return tma_smem_bytes(storage, L, ty) <= 220 * 1024;
}

// Whether a Potts state set can be staged by TMA: 16-byte aligned plane
// bases and row strides.
bool potts_tma_eligible(const Grid& G, int storage, const PottsStateV& s) {
    const size_t es = dtype_size(storage);
    if ((G.pitch * es) % 16 || (G.pitch * 4) % 16) return false;
    auto al = [](const void* p) { return ((uintptr_t)p % 16) == 0; };
    return al(s.u) && al(s.qx) && al(s.qy) && al(s.p) && al(s.ps);
}

cudaError_t potts_tma_maps(const Grid& G, int L, int storage, const PottsStateV& s, int ty,
                           PottsTmaMaps& m) {
    const int es = (int)dtype_size(storage);
    const int bxs = es == 4 ? 40 : 48;
    const int by = ty + 3;
    cudaError_t e;
    if ((e = encode_tma_3d(&m.qx, s.qx, es, G.W, G.H, L, G.pitch, bxs, by)) != cudaSuccess)
        return e;
    if ((e = encode_tma_3d(&m.qy, s.qy, es, G.W, G.H, L, G.pitch, bxs, by)) != cudaSuccess)
        return e;
    if ((e = encode_tma_3d(&m.p, s.p, es, G.W, G.H, L, G.pitch, bxs, by)) != cudaSuccess)
        return e;
    if ((e = encode_tma_3d(&m.u, s.u, 4, G.W, G.H, L, G.pitch, 40, by)) != cudaSuccess) return e;
    if ((e = encode_tma_3d(&m.ps, s.ps, es, G.W, G.H, 1, G.pitch, bxs, by)) != cudaSuccess)
        return e;
    m.ty = ty;
    return cudaSuccess;
}

template <typename S, bool ANISO, int TY>
static cudaError_t launch_tma(const PottsProblem& P, const PottsState<S>& b, const AdmmCoef& K,
                              const PottsTmaMaps& m, int* err, cudaStream_t st) {
    using Lay = PottsTmaLayout<S, TY>;
    const size_t dyn = Lay::dyn_bytes(P.L);
    auto kern = k_potts_admm_tma<S, ANISO, TY>;
    static size_t configured = 0;
    if (dyn > configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)dyn);
        if (e != cudaSuccess) return e;
        configured = dyn;
    }
    const dim3 grid((P.g.W + 31) / 32, (P.g.H + TY - 1) / TY);
    kern<<<grid, dim3(32, 8), dyn, st>>>(P, b, K, m.qx, m.qy, m.p, m.u, m.ps, err);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t potts_admm_tma_s(const PottsProblem& P, const PottsStateV& b, bool aniso,
                                    const AdmmCoef& K, const PottsTmaMaps& m, int* err,
                                    cudaStream_t st) {
    const PottsState<S> B = b.as<S>();
    if (m.ty == 32)
        return aniso ? launch_tma<S, true, 32>(P, B, K, m, err, st)
                     : launch_tma<S, false, 32>(P, B, K, m, err, st);
    return aniso ? launch_tma<S, true, 16>(P, B, K, m, err, st)
                 : launch_tma<S, false, 16>(P, B, K, m, err, st);
}

cudaError_t potts_admm_tma_step(int storage, const PottsProblem& P, const PottsStateV& b,
                                bool aniso, const AdmmCoef& K, const PottsTmaMaps& src_maps,
                                int* err, cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return potts_admm_tma_s<float>(P, b, aniso, K, src_maps, err, st);
        case CMF_F16: return potts_admm_tma_s<__half>(P, b, aniso, K, src_maps, err, st);
        default: return potts_admm_tma_s<__nv_bfloat16>(P, b, aniso, K, src_maps, err, st);
    }
}

}  // namespace cmf
