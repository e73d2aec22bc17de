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

#ifdef CMF_FAULT_INJECTION
// Fault-injection test build only (never in the library the product loads):
// extra bytes the p_s stage's barrier expects beyond what its copy delivers.
// With a non-zero value that barrier's phase cannot complete, the bounded
// wait runs out, the kernel records kErrWaitTimeout and returns; nothing
// faults and no copy is left in flight.
__device__ unsigned int g_inject_extra_tx = 0;
#define CMF_PS_EXTRA_TX g_inject_extra_tx
#else
#define CMF_PS_EXTRA_TX 0u
#endif

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
    // p_s is float32 for every flow storage: staged like u
    static constexpr uint32_t PS_BYTES = (uint32_t)BY * BXU * 4u;
    // + 128: the kernel rounds the dynamic shared-memory base up to 128 bytes
    static size_t dyn_bytes(int L) { return 2 * STAGE + FU + (size_t)L * TY * 32 * 4 + 128; }
};

template <typename S>
__device__ __forceinline__ float sload(const S* p) {
    return Store<S>::ldw(p);
}

}  // namespace

template <typename S, bool ANISO, int TY>
__global__ void __launch_bounds__(256, TY <= 16 ? 4 : 2)
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
    constexpr int GW = TX + 2, GH = TY + 2;  // g cells: rows y0-1.., cols x0-1..
    constexpr int QW = TX + 1, QH = TY + 1;  // q cells: rows y0-1.., cols x0-1..
    constexpr int NG = (GW * GH + 255) / 256;
    constexpr int NQ = (QW * QH + 255) / 256;
    __shared__ __align__(8) uint64_t bar[3];
    // cell arrays padded to whole multiples of the block so every thread owns
    // NG / NQ slots; the padding slots are computed and never read
    __shared__ float g_s[NG * 256];
    __shared__ float qnx[NQ * 256];
    __shared__ float qny[NQ * 256];
    extern __shared__ __align__(128) unsigned char dsm_raw[];
    // round up to 128 bytes by pointer arithmetic (keeps the shared space)
    unsigned char* dsm = dsm_raw + ((128u - (smem_u32(dsm_raw) & 127u)) & 127u);
    float* ps_s = reinterpret_cast<float*>(dsm + 2 * Lay::STAGE);
    // the p_s box starts XO - XU columns later than the S boxes
    const float* sps = ps_s - (XO - XU);
    float* v_s = reinterpret_cast<float*>(dsm + 2 * Lay::STAGE + Lay::FU);

    const Grid G = P.g;
    const int L = P.L;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

    auto issue = [&](int l, int s) {
        unsigned char* d = dsm + s * Lay::STAGE;
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
        mbar_arrive_expect_tx(&bar[2], Lay::PS_BYTES + CMF_PS_EXTRA_TX);
        tma_load_3d(ps_s, &mps, &bar[2], x0 - XU, y0 - 2, 0);
        issue(0, 0);
        if (L > 1) issue(1, 1);
    }

    // ---- per-thread cell data, the same for every label ----------------------
    // g cells: staged offset (the u box is addressed through a pointer shifted
    // by XO - XU columns) and the 0/1 weights of the far-boundary terms
    int g_off[NG], g_uoff[NG];
    float g_mx[NG], g_my[NG];
#pragma unroll
    for (int n = 0; n < NG; ++n) {
        const int i = tid + 256 * n;
        const int gy = i < GW * GH ? i / GW : 0, gx = i < GW * GH ? i - gy * GW : 1;
        const int r = y0 - 1 + gy, c = x0 - 1 + gx;
        g_off[n] = (gy + 1) * BXS + gx - 1 + XO;
        g_uoff[n] = (gy + 1) * BXU + gx - 1 + XO;
        g_mx[n] = c < G.W - 1 ? 1.f : 0.f;
        g_my[n] = r < G.H - 1 ? 1.f : 0.f;
    }
    // q cells: staged offset, g offset, weights (times 1/a), alpha, in-grid
    // flag, output pointers of the tile part (null: halo or outside)
    int q_off[NQ], q_goff[NQ];
    float q_mx[NQ], q_my[NQ], q_al[NQ];
    bool q_in[NQ];
    long long q_k[NQ];
#pragma unroll
    for (int n = 0; n < NQ; ++n) {
        const int i = tid + 256 * n;
        const bool cell = i < QW * QH;
        const int qy_ = cell ? i / QW : 1, qx_ = cell ? i - qy_ * QW : 1;
        const int r = y0 - 1 + qy_, c = x0 - 1 + qx_;
        const bool in = cell && r >= 0 && r < G.H && c >= 0 && c < G.W;
        q_in[n] = in;
        q_off[n] = (qy_ + 1) * BXS + qx_ - 1 + XO;
        q_goff[n] = qy_ * GW + qx_;
        q_mx[n] = c < G.W - 1 ? K.inv_a : 0.f;
        q_my[n] = r < G.H - 1 ? K.inv_a : 0.f;
        q_al[n] = in ? P.alpha.at(G.idx(r, c)) : 0.f;
        q_k[n] = (in && qy_ >= 1 && qx_ >= 1) ? (long long)G.idx(r, c) : -1;
    }
    // own pixels
    long long o_k[ROWS];
    float o_mx[ROWS], o_my[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
        const int r = y0 + threadIdx.y + 8 * j, c = x0 + threadIdx.x;
        o_k[j] = (r < G.H && c < G.W) ? (long long)G.idx(r, c) : -1;
        o_mx[j] = c < G.W - 1 ? 1.f : 0.f;
        o_my[j] = r < G.H - 1 ? 1.f : 0.f;
    }

    bool ok = mbar_wait_bounded(&bar[2], 0, kWaitLimitCycles);
    float accd[ROWS], accp[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) accd[j] = accp[j] = 0.f;

    // warps whose slots of the last round all lie past the cell count skip it
    const bool g_tail = (tid & ~31) < GW * GH - 256 * (NG - 1);
    const bool q_tail = (tid & ~31) < QW * QH - 256 * (NQ - 1);
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
        const int s = l & 1;
        const unsigned char* stg = dsm + s * Lay::STAGE;
        const S* sqx = reinterpret_cast<const S*>(stg);
        const S* sqy = reinterpret_cast<const S*>(stg + Lay::FS);
        const S* sp = reinterpret_cast<const S*>(stg + 2 * Lay::FS);
        // the u box starts XO - XU columns later than the S boxes
        const float* su = reinterpret_cast<const float*>(stg + 3 * Lay::FS) - (XO - XU);
        ok = ok && mbar_wait_bounded(&bar[s], (l >> 1) & 1, kWaitLimitCycles);
        if (__syncthreads_or(!ok)) {
            // a TMA stage never arrived: flag it, give in-flight copies a
            // bounded chance to land in this block's shared memory, return
            if (tid == 0) {
                atomicExch(err, kErrWaitTimeout);
                mbar_wait_bounded(&bar[0], (l >> 1) & 1, kWaitLimitCycles);
                if (L > 1) mbar_wait_bounded(&bar[1], (l >> 1) & 1, kWaitLimitCycles);
            }
            return;
        }
        const size_t lo = (size_t)l * G.plane;
        S* qx_out = s1.qx + lo;
        S* qy_out = s1.qy + lo;
        S* p_out = s1.p + lo;

        // g_l = div q_l + p_l - p_s - u_l / c (zero-filled outside the grid)
#pragma unroll
        for (int n = 0; n < NG; ++n) {
            if (n == NG - 1 && !g_tail) break;
            const int o = g_off[n];
            float dv = g_mx[n] * sload(sqx + o);
            dv -= sload(sqx + o - 1);
            dv += g_my[n] * sload(sqy + o);
            dv -= sload(sqy + o - BXS);
            g_s[tid + 256 * n] =
                dv + sload(sp + o) - sps[g_uoff[n]] - su[g_uoff[n]] * K.inv_c;
        }
        __syncthreads();

        // q_l^{k+1} = P_alpha(q_l + grad g_l / a); 0 outside the grid
#pragma unroll
        for (int n = 0; n < NQ; ++n) {
            if (n == NQ - 1 && !q_tail) break;
            const int o = q_off[n], go = q_goff[n];
            const float gc = g_s[go];
            float tx = sload(sqx + o) + (g_s[go + 1] - gc) * q_mx[n];
            float ty = sload(sqy + o) + (g_s[go + GW] - gc) * q_my[n];
            project_alpha<ANISO>(tx, ty, q_al[n]);
            tx = q_in[n] ? St::rt(tx) : 0.f;
            ty = q_in[n] ? St::rt(ty) : 0.f;
            if (q_k[n] >= 0) {
                St::st(qx_out + q_k[n], tx);
                St::st(qy_out + q_k[n], ty);
            }
            qnx[tid + 256 * n] = tx;
            qny[tid + 256 * n] = ty;
        }
        __syncthreads();

        // d_l, p_l^{k+1}, the p_s terms and v_l on the tile
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
            const int qi = (ly + 1) * QW + lx + 1;
            float d = o_mx[j] * qnx[qi];
            d -= qnx[qi - 1];
            d += o_my[j] * qny[qi];
            d -= qny[qi - QW];
            const int so = (ly + 2) * BXS + lx + XO;
            const float ps0 = sps[(ly + 2) * BXU + lx + XO];
            const float p0 = sload(sp + so);
            const float u0 = su[(ly + 2) * BXU + lx + XO];
            const bool own = o_k[j] >= 0;
            const float cl = potts_cost(P, l, own ? (size_t)o_k[j] : 0);
            float v;
            const float p1 = potts_label_pu<S>(K, g_s[(ly + 1) * GW + lx + 1], d, p0, ps0, u0, cl,
                                               accd[j], accp[j], v);
            if (own) St::st(p_out + o_k[j], p1);
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
        const float ps0 = sps[(ly + 2) * BXU + lx + XO];
        ps1[j] = potts_ps_update(K, ps0, accd[j], accp[j]);
        if (o_k[j] >= 0) s1.ps[o_k[j]] = ps1[j];
    }
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
        float* u_out = s1.u + (size_t)l * G.plane;
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            const int ly = threadIdx.y + 8 * j, lx = threadIdx.x;
            if (o_k[j] >= 0) u_out[o_k[j]] = v_s[(l * TY + ly) * TX + lx] + K.cu * ps1[j];
        }
    }
}

// Shared memory one block of the TMA kernel needs (static + dynamic).
static size_t tma_smem_bytes(int storage, int L, int ty) {
    const size_t ng = ((size_t)(ty + 2) * 34 + 255) / 256, nq = ((size_t)(ty + 1) * 33 + 255) / 256;
    const size_t stat = (ng + 2 * nq) * 256 * 4 + 64;
    size_t dyn;
    if (storage == CMF_F32)
        dyn = ty == 32 ? PottsTmaLayout<float, 32>::dyn_bytes(L)
                       : (ty == 8 ? PottsTmaLayout<float, 8>::dyn_bytes(L)
                                  : PottsTmaLayout<float, 16>::dyn_bytes(L));
    else
        dyn = ty == 32 ? PottsTmaLayout<__half, 32>::dyn_bytes(L)
                       : (ty == 8 ? PottsTmaLayout<__half, 8>::dyn_bytes(L)
                                  : PottsTmaLayout<__half, 16>::dyn_bytes(L));
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
    if ((e = encode_tma_3d(&m.ps, s.ps, 4, G.W, G.H, 1, G.pitch, 40, by)) != cudaSuccess) return e;
    m.ty = ty;
    return cudaSuccess;
}

// Raise the kernel's dynamic shared-memory limit to what L labels need.
template <typename S, bool ANISO, int TY>
static cudaError_t configure_tma(size_t dyn) {
    static std::atomic<long long> memo[kMaxDevices];  // limit set on each device
    return raise_dyn_smem(memo, k_potts_admm_tma<S, ANISO, TY>, dyn);
}

// Warps of this kernel resident per SM for L labels (0 on error).
template <typename S, bool ANISO, int TY>
static int resident_warps(int L) {
    const size_t dyn = PottsTmaLayout<S, TY>::dyn_bytes(L);
    int blocks = 0;
    if (configure_tma<S, ANISO, TY>(dyn) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_potts_admm_tma<S, ANISO, TY>,
                                                      256, dyn) != cudaSuccess)
        return 0;
    return blocks * 8;
}

template <typename S, bool ANISO>
static int auto_ty(int L) {
    if (!potts_tma_fits(sizeof(S) == 4 ? CMF_F32 : CMF_F16, L, 16)) return 8;
    return resident_warps<S, ANISO, 8>(L) > resident_warps<S, ANISO, 16>(L) ? 8 : 16;
}

int potts_tma_auto_ty(int storage, bool aniso, int L) {
    switch (storage) {
        case CMF_F32: return aniso ? auto_ty<float, true>(L) : auto_ty<float, false>(L);
        case CMF_F16: return aniso ? auto_ty<__half, true>(L) : auto_ty<__half, false>(L);
        default:
            return aniso ? auto_ty<__nv_bfloat16, true>(L) : auto_ty<__nv_bfloat16, false>(L);
    }
}

template <typename S, bool ANISO, int TY>
static cudaError_t launch_tma(const PottsProblem& P, const PottsState<S>& b, const AdmmCoef& K,
                              const PottsTmaMaps& m, int* err, cudaStream_t st) {
    using Lay = PottsTmaLayout<S, TY>;
    const size_t dyn = Lay::dyn_bytes(P.L);
    auto kern = k_potts_admm_tma<S, ANISO, TY>;
    cudaError_t e = configure_tma<S, ANISO, TY>(dyn);
    if (e != cudaSuccess) return e;
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
    if (m.ty == 8)
        return aniso ? launch_tma<S, true, 8>(P, B, K, m, err, st)
                     : launch_tma<S, false, 8>(P, B, K, m, err, st);
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

#ifdef CMF_FAULT_INJECTION
// Test hook of the fault-injection build: every later Potts TMA launch on the
// current device expects `bytes` more on its p_s barrier than its copy
// delivers (0 switches it off).
extern "C" cmf_status cmf_debug_inject_tx_mismatch(unsigned int bytes) {
    return cudaMemcpyToSymbol(cmf::g_inject_extra_tx, &bytes, sizeof(bytes)) == cudaSuccess
               ? CMF_OK
               : CMF_ECUDA;
}
#endif
