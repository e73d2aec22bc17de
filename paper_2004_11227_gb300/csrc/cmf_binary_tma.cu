// Binary ADMM iteration (Eq. rpADMMI / Eq. rpADMMII) as a persistent kernel
// with TMA-staged tiles.
//
// Each block walks output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// The five state planes it reads with a halo (q_x, q_y, p_s, p_t, u) arrive
// as TMA boxes in one of two shared-memory stages, so tile k+2 is in flight
// while tile k is computed.  Shared-memory offsets of a thread's cells are
// the same for every tile and are computed once.
//
// Staged box: rows y0-2 .. y0+TY, columns x0-XO .. x0-XO+BX-1 (XO = 4 for
// 4-byte elements, 8 for 2-byte ones: 16-byte aligned box starts); elements
// outside the grid read as zero.
#include "cmf_kernels.cuh"
#include "cmf_tma.cuh"

namespace cmf {

namespace {

constexpr int align128b(int b) { return (b + 127) / 128 * 128; }

template <typename S, int TY>
struct BinTmaLayout {
    static constexpr int BY = TY + 3;
    static constexpr int XO = sizeof(S) == 4 ? 4 : 8;
    static constexpr int BXS = sizeof(S) == 4 ? 40 : 48;
    static constexpr int XU = 4, BXU = 40;
    static constexpr int FS = align128b(BY * BXS * (int)sizeof(S));
    static constexpr int FU = align128b(BY * BXU * 4);
    static constexpr int STAGE = 4 * FS + FU;
    static constexpr uint32_t TX_BYTES = 4u * BY * BXS * sizeof(S) + (uint32_t)BY * BXU * 4u;
    static constexpr size_t DYN = 2 * (size_t)STAGE + 128;
};

template <typename S>
__device__ __forceinline__ float bload(const S* p) {
    return Store<S>::ldw(p);
}

}  // namespace

template <typename S, bool ANISO, int TY>
__global__ void __launch_bounds__(256, 4)
    k_binary_admm_tma(BinProblem P, BinState<S> s1, AdmmCoef K,
                      const __grid_constant__ CUtensorMap mqx,
                      const __grid_constant__ CUtensorMap mqy,
                      const __grid_constant__ CUtensorMap mps,
                      const __grid_constant__ CUtensorMap mpt,
                      const __grid_constant__ CUtensorMap mu, int* err) {
    using Lay = BinTmaLayout<S, TY>;
    using St = Store<S>;
    constexpr int TX = 32, ROWS = TY / 8;
    constexpr int BXS = Lay::BXS, BXU = Lay::BXU, XO = Lay::XO, XU = Lay::XU;
    constexpr int GW = TX + 2, GH = TY + 2;
    constexpr int QW = TX + 1, QH = TY + 1;
    constexpr int NG = (GW * GH + 255) / 256;
    constexpr int NQ = (QW * QH + 255) / 256;
    __shared__ __align__(8) uint64_t bar[2];
    // cell arrays padded to whole multiples of the block; padding slots are
    // computed and never read
    __shared__ float g_s[NG * 256];
    __shared__ float qnx[NQ * 256];
    __shared__ float qny[NQ * 256];
    extern __shared__ __align__(128) unsigned char dsm_raw[];
    // round up to 128 bytes by pointer arithmetic (keeps the shared space)
    unsigned char* dsm = dsm_raw + ((128u - (smem_u32(dsm_raw) & 127u)) & 127u);

    const Grid G = P.g;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int ntx = (G.W + TX - 1) / TX;
    const int ntiles = ntx * ((G.H + TY - 1) / TY);

    auto issue = [&](int t, int s) {
        const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
        unsigned char* d = dsm + s * Lay::STAGE;
        mbar_arrive_expect_tx(&bar[s], Lay::TX_BYTES);
        tma_load_3d(d, &mqx, &bar[s], x0 - XO, y0 - 2, 0);
        tma_load_3d(d + Lay::FS, &mqy, &bar[s], x0 - XO, y0 - 2, 0);
        tma_load_3d(d + 2 * Lay::FS, &mps, &bar[s], x0 - XO, y0 - 2, 0);
        tma_load_3d(d + 3 * Lay::FS, &mpt, &bar[s], x0 - XO, y0 - 2, 0);
        tma_load_3d(d + 4 * Lay::FS, &mu, &bar[s], x0 - XU, y0 - 2, 0);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int t0 = blockIdx.x, dt = gridDim.x;
    if (tid == 0) {
        if (t0 < ntiles) issue(t0, 0);
        if (t0 + dt < ntiles) issue(t0 + dt, 1);
    }

    // tile-invariant cell data: tile-relative coordinates and shared offsets
    int g_off[NG], g_uoff[NG], g_r[NG], g_c[NG];
#pragma unroll
    for (int n = 0; n < NG; ++n) {
        const int i = tid + 256 * n;
        const int gy = i < GW * GH ? i / GW : 0, gx = i < GW * GH ? i - gy * GW : 1;
        g_off[n] = (gy + 1) * BXS + gx - 1 + XO;
        g_uoff[n] = (gy + 1) * BXU + gx - 1 + XO;
        g_r[n] = gy - 1;
        g_c[n] = gx - 1;
    }
    int q_off[NQ], q_goff[NQ], q_r[NQ], q_c[NQ];
    bool q_cell[NQ];
#pragma unroll
    for (int n = 0; n < NQ; ++n) {
        const int i = tid + 256 * n;
        q_cell[n] = i < QW * QH;
        const int qy_ = q_cell[n] ? i / QW : 1, qx_ = q_cell[n] ? i - qy_ * QW : 1;
        q_off[n] = (qy_ + 1) * BXS + qx_ - 1 + XO;
        q_goff[n] = qy_ * GW + qx_;
        q_r[n] = qy_ - 1;
        q_c[n] = qx_ - 1;
    }

    // warps whose slots of the last round all lie past the cell count skip it
    const bool g_tail = (tid & ~31) < GW * GH - 256 * (NG - 1);
    const bool q_tail = (tid & ~31) < QW * QH - 256 * (NQ - 1);
#pragma unroll 1
    for (int t = t0, k = 0; t < ntiles; t += dt, ++k) {
        const int s = k & 1;
        const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
        const unsigned char* stg = dsm + s * Lay::STAGE;
        const S* sqx = reinterpret_cast<const S*>(stg);
        const S* sqy = reinterpret_cast<const S*>(stg + Lay::FS);
        const S* sps = reinterpret_cast<const S*>(stg + 2 * Lay::FS);
        const S* spt = reinterpret_cast<const S*>(stg + 3 * Lay::FS);
        const float* su = reinterpret_cast<const float*>(stg + 4 * Lay::FS) - (XO - XU);
        const bool ok = mbar_wait_bounded(&bar[s], (k >> 1) & 1, kWaitLimitCycles);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(err, kErrWaitTimeout);
                mbar_wait_bounded(&bar[s ^ 1], ((k + 1) >> 1) & 1, kWaitLimitCycles);
            }
            return;
        }

        // g = div q + p_t - p_s - u / c on rows y0-1..y0+TY, cols x0-1..x0+TX
#pragma unroll
        for (int n = 0; n < NG; ++n) {
            if (n == NG - 1 && !g_tail) break;
            const int o = g_off[n];
            const int r = y0 + g_r[n], c = x0 + g_c[n];
            float dv = c < G.W - 1 ? bload(sqx + o) : 0.f;
            dv -= bload(sqx + o - 1);
            dv += r < G.H - 1 ? bload(sqy + o) : 0.f;
            dv -= bload(sqy + o - BXS);
            g_s[tid + 256 * n] = dv + bload(spt + o) - bload(sps + o) - su[g_uoff[n]] * K.inv_c;
        }
        __syncthreads();

        // q^{k+1} = P_alpha(q + grad g / a) on rows y0-1.., cols x0-1..
#pragma unroll
        for (int n = 0; n < NQ; ++n) {
            if (n == NQ - 1 && !q_tail) break;
            const int o = q_off[n], go = q_goff[n];
            const int r = y0 + q_r[n], c = x0 + q_c[n];
            const bool in = q_cell[n] && r >= 0 && r < G.H && c >= 0 && c < G.W;
            const size_t kk = in ? G.idx(r, c) : 0;
            const float gc = g_s[go];
            float tx = bload(sqx + o) + (c < G.W - 1 ? (g_s[go + 1] - gc) * K.inv_a : 0.f);
            float ty = bload(sqy + o) + (r < G.H - 1 ? (g_s[go + GW] - gc) * K.inv_a : 0.f);
            project_alpha<ANISO>(tx, ty, P.alpha.at(kk));
            tx = in ? St::rt(tx) : 0.f;
            ty = in ? St::rt(ty) : 0.f;
            if (in && q_r[n] >= 0 && q_c[n] >= 0) {
                St::st(s1.qx + kk, tx);
                St::st(s1.qy + kk, ty);
            }
            qnx[tid + 256 * n] = tx;
            qny[tid + 256 * n] = ty;
        }
        __syncthreads();

        // d = div q^{k+1}, p^{k+1}, u^{k+1} on the tile
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
            const int r = y0 + ly, c = x0 + lx;
            if (r < G.H && c < G.W) {
                const size_t kk = G.idx(r, c);
                const int qi = (ly + 1) * QW + lx + 1;
                float d = 0.f;
                if (c < G.W - 1) d += qnx[qi];
                d -= qnx[qi - 1];
                if (r < G.H - 1) d += qny[qi];
                d -= qny[qi - QW];
                const int so = (ly + 2) * BXS + lx + XO;
                const float ps0 = bload(sps + so), pt0 = bload(spt + so);
                const float u0 = su[(ly + 2) * BXU + lx + XO];
                float ps1, pt1, u1;
                binary_pu<S>(K, g_s[(ly + 1) * GW + lx + 1], d, ps0, pt0, u0, __ldg(P.Cs + kk),
                             __ldg(P.Ct + kk), ps1, pt1, u1);
                St::st(s1.ps + kk, ps1);
                St::st(s1.pt + kk, pt1);
                s1.u[kk] = u1;
            }
        }
        __syncthreads();
        if (tid == 0 && t + 2 * dt < ntiles) {
            fence_proxy_async_smem();
            issue(t + 2 * dt, s);
        }
    }
}

bool binary_tma_eligible(const Grid& G, int storage, const BinStateV& s) {
    const size_t es = dtype_size(storage);
    if ((G.pitch * es) % 16 || (G.pitch * 4) % 16) return false;
    auto al = [](const void* p) { return ((uintptr_t)p % 16) == 0; };
    return al(s.u) && al(s.qx) && al(s.qy) && al(s.ps) && al(s.pt);
}

cudaError_t binary_tma_maps(const Grid& G, int storage, const BinStateV& s, int ty,
                            BinTmaMaps& m) {
    const int es = (int)dtype_size(storage);
    const int bxs = es == 4 ? 40 : 48;
    const int by = ty + 3;
    cudaError_t e;
    if ((e = encode_tma_3d(&m.qx, s.qx, es, G.W, G.H, 1, G.pitch, bxs, by)) != cudaSuccess)
        return e;
    if ((e = encode_tma_3d(&m.qy, s.qy, es, G.W, G.H, 1, G.pitch, bxs, by)) != cudaSuccess)
        return e;
    if ((e = encode_tma_3d(&m.ps, s.ps, es, G.W, G.H, 1, G.pitch, bxs, by)) != cudaSuccess)
        return e;
    if ((e = encode_tma_3d(&m.pt, s.pt, es, G.W, G.H, 1, G.pitch, bxs, by)) != cudaSuccess)
        return e;
    if ((e = encode_tma_3d(&m.u, s.u, 4, G.W, G.H, 1, G.pitch, 40, by)) != cudaSuccess) return e;
    m.ty = ty;
    return cudaSuccess;
}

template <typename S, bool ANISO, int TY>
static cudaError_t launch_bin_tma(const BinProblem& P, const BinState<S>& b, const AdmmCoef& K,
                                  const BinTmaMaps& m, int* err, cudaStream_t st) {
    using Lay = BinTmaLayout<S, TY>;
    auto kern = k_binary_admm_tma<S, ANISO, TY>;  // static smem: (NG + 2 NQ) x 256 floats
    static std::atomic<long long> memo[kMaxDevices];  // resident blocks per device
    long long resident = 0;
    {
        const cudaError_t e = per_device(
            memo,
            [&](int dev, long long& v) -> cudaError_t {
                cudaError_t e2 = cudaFuncSetAttribute(
                    kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::DYN);
                if (e2 != cudaSuccess) return e2;
                int sms = 0, blocks_per_sm = 0;
                if ((e2 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) !=
                    cudaSuccess)
                    return e2;
                if ((e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, 256,
                                                                         Lay::DYN)) !=
                    cudaSuccess)
                    return e2;
                v = (long long)sms * (blocks_per_sm > 0 ? blocks_per_sm : 1);
                return cudaSuccess;
            },
            resident);
        if (e != cudaSuccess) return e;
    }
    const int ntiles = ((P.g.W + 31) / 32) * ((P.g.H + TY - 1) / TY);
    int grid = (int)resident;
    if (grid > ntiles) grid = ntiles;
    kern<<<grid, dim3(32, 8), Lay::DYN, st>>>(P, b, K, m.qx, m.qy, m.ps, m.pt, m.u, err);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t binary_tma_s(const BinProblem& P, const BinStateV& b, bool aniso,
                                const AdmmCoef& K, const BinTmaMaps& m, int* err,
                                cudaStream_t st) {
    const BinState<S> B = b.as<S>();
    if (m.ty == 8)
        return aniso ? launch_bin_tma<S, true, 8>(P, B, K, m, err, st)
                     : launch_bin_tma<S, false, 8>(P, B, K, m, err, st);
    if (m.ty == 32)
        return aniso ? launch_bin_tma<S, true, 32>(P, B, K, m, err, st)
                     : launch_bin_tma<S, false, 32>(P, B, K, m, err, st);
    return aniso ? launch_bin_tma<S, true, 16>(P, B, K, m, err, st)
                 : launch_bin_tma<S, false, 16>(P, B, K, m, err, st);
}

cudaError_t binary_admm_tma_step(int storage, const BinProblem& P, const BinStateV& b,
                                 bool aniso, const AdmmCoef& K, const BinTmaMaps& src_maps,
                                 int* err, cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return binary_tma_s<float>(P, b, aniso, K, src_maps, err, st);
        case CMF_F16: return binary_tma_s<__half>(P, b, aniso, K, src_maps, err, st);
        default: return binary_tma_s<__nv_bfloat16>(P, b, aniso, K, src_maps, err, st);
    }
}

}  // namespace cmf
