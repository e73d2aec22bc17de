// Binary ADMM iteration by warp strips (Eq. rpADMMII, Eq. rpADMMI, pADMM-TY
// Eq. ADMM:Tai_yuan).
//
// Work unit: one warp, a strip of 64 columns (two adjacent columns per lane)
// and a band of R output rows, streamed top-down.  Step t holds rows t and
// t+1 of the state in registers while row t+2 is in flight, makes g of row
// t+1, the new flow q of row t (column neighbours by warp shuffles), its
// divergence, and the pointwise p_s, p_t, u update of row t.  Lanes cover
// columns cs-2 .. cs+61 and own the output columns cs .. cs+59.
#include <climits>

#include "cmf_kernels.cuh"
#include "cmf_strip.cuh"

namespace cmf {

using strip::kStripOut;
using strip::kStripWarps;
using strip::Pair;
using strip::project_sel;

namespace {

// State values of one row at this lane's column pair.
template <typename S>
struct BinRow {
    typename Pair<S>::T qx, qy, ps, pt;
    float2 u;
};

}  // namespace

template <typename S, bool ANISO>
__global__ void __launch_bounds__(kStripWarps * 32, 8)
    k_binary_strip(BinProblem P, BinState<S> s0, BinState<S> s1, AdmmCoef K, int R,
                   int nstrips, int nitems) {
    using St = Store<S>;
    using PS = Pair<S>;
    using PF = Pair<float>;
    const int lane = threadIdx.x & 31;
    const Grid G = P.g;
    const unsigned full = 0xffffffffu;

    for (int item = blockIdx.x * kStripWarps + (threadIdx.x >> 5); item < nitems;
         item += gridDim.x * kStripWarps) {
        const int cs = (item % nstrips) * kStripOut;
        const int r0 = (item / nstrips) * R;
        const int r1 = min(r0 + R, G.H);
        const int c = cs - 2 + 2 * lane;  // even column of the pair (W is even)
        const bool colin = c >= 0 && c < G.W;
        const bool own = colin && lane >= 1 && lane <= 30;
        const float mxo = c + 1 < G.W - 1 ? 1.f : 0.f;  // odd column is not the last

        auto ok_row = [&](int r) { return colin && r >= 0 && r < G.H; };
        auto row = [&](int r, BinRow<S>& x) {
            const bool ok = ok_row(r);
            const int o = r * G.pitch + c;
            x.qx = ok ? PS::ld(s0.qx + o) : PS::zero();
            x.qy = ok ? PS::ld(s0.qy + o) : PS::zero();
            x.ps = ok ? PS::ld(s0.ps + o) : PS::zero();
            x.pt = ok ? PS::ld(s0.pt + o) : PS::zero();
            x.u = ok ? PF::ld(s0.u + o) : PF::zero();
        };
        auto ld_f = [&](const float* base, int r) {
            return ok_row(r) ? PF::ld(base + r * G.pitch + c) : PF::zero();
        };
        auto ld_al = [&](int r) {
            if (!P.alpha.plane) return make_float2(P.alpha.value, P.alpha.value);
            return ld_f(P.alpha.plane, r);
        };
        auto row_w = [&](int r) { return r < G.H - 1 ? 1.f : 0.f; };
        // g = div q + p_t - p_s - u / c at row r, given the row above's q_y
        auto g_of = [&](const BinRow<S>& x, float2 qy_up, int r) {
            const float2 qx = PS::f2(x.qx), qy = PS::f2(x.qy);
            const float2 ps = PS::f2(x.ps), pt = PS::f2(x.pt);
            const float qx_left = __shfl_up_sync(full, qx.y, 1);
            const float wy = row_w(r);
            float2 g;
            g.x = qx.x - qx_left + wy * qy.x - qy_up.x + pt.x - ps.x - x.u.x * K.inv_c;
            g.y = mxo * qx.y - qx.x + wy * qy.y - qy_up.y + pt.y - ps.y - x.u.y * K.inv_c;
            return g;
        };

        BinRow<S> a, b, nx;
        const int rm2 = r0 - 2;
        const float2 qy_m2 =
            PS::f2(ok_row(rm2) ? PS::ld(s0.qy + rm2 * G.pitch + c) : PS::zero());
        row(r0 - 1, a);
        row(r0, b);
        float2 g_t = g_of(a, qy_m2, r0 - 1);
        float2 qyn_up = make_float2(0.f, 0.f);  // new q_y of the row above
        float2 al_t = ld_al(r0 - 1), cs_t = PF::zero(), ct_t = PF::zero();
        float2 al_n = al_t, cs_n = cs_t, ct_n = ct_t;
#pragma unroll 1
        for (int t = r0 - 1; t < r1; ++t) {
            if (t + 2 <= r1) row(t + 2, nx);  // in flight during this row
            if (t + 1 < r1) {
                al_n = ld_al(t + 1);
                cs_n = ld_f(P.Cs, t + 1);
                ct_n = ld_f(P.Ct, t + 1);
            }
            const float2 g_n = g_of(b, PS::f2(a.qy), t + 1);  // g at row t+1

            // q^{k+1} = P_alpha(q + grad g / a) at row t
            const float g_r = __shfl_down_sync(full, g_t.x, 1);  // g(t, c+2)
            const float my = row_w(t) * K.inv_a;
            const float2 qx = PS::f2(a.qx), qy = PS::f2(a.qy);
            float tx_e = qx.x + (g_t.y - g_t.x) * K.inv_a;
            float tx_o = qx.y + (g_r - g_t.y) * (mxo * K.inv_a);
            float ty_e = qy.x + (g_n.x - g_t.x) * my;
            float ty_o = qy.y + (g_n.y - g_t.y) * my;
            project_sel<ANISO>(tx_e, ty_e, al_t.x);
            project_sel<ANISO>(tx_o, ty_o, al_t.y);
            const bool in = colin && t >= 0;  // t < r1 <= H
            tx_e = in ? St::rt(tx_e) : 0.f;
            tx_o = in ? St::rt(tx_o) : 0.f;
            ty_e = in ? St::rt(ty_e) : 0.f;
            ty_o = in ? St::rt(ty_o) : 0.f;

            if (t >= r0) {
                // d = div q^{k+1}, then p_s, p_t, u at row t
                const float txl = __shfl_up_sync(full, tx_o, 1);  // new q_x at c-1
                const float wy = row_w(t);
                const float d_e = tx_e - txl + wy * ty_e - qyn_up.x;
                const float d_o = mxo * tx_o - tx_e + wy * ty_o - qyn_up.y;
                const float2 ps = PS::f2(a.ps), pt = PS::f2(a.pt);
                float ps_e, pt_e, u_e, ps_o, pt_o, u_o;
                binary_pu<S>(K, g_t.x, d_e, ps.x, pt.x, a.u.x, cs_t.x, ct_t.x, ps_e, pt_e, u_e);
                binary_pu<S>(K, g_t.y, d_o, ps.y, pt.y, a.u.y, cs_t.y, ct_t.y, ps_o, pt_o, u_o);
                if (own) {
                    const int o = t * G.pitch + c;
                    PS::st(s1.qx + o, tx_e, tx_o);
                    PS::st(s1.qy + o, ty_e, ty_o);
                    PS::st(s1.ps + o, ps_e, ps_o);
                    PS::st(s1.pt + o, pt_e, pt_o);
                    PF::st(s1.u + o, u_e, u_o);
                }
            }
            qyn_up = make_float2(ty_e, ty_o);
            a = b;
            b = nx;
            g_t = g_n;
            al_t = al_n;
            cs_t = cs_n;
            ct_t = ct_n;
        }
    }
}

// ---- rPDRQ by warp strips (Eq. iteration:quadratic:seg) -------------------
//
// One iteration: b = -sigma (div qbar + pbar_t - pbar_s); the symmetric
// red-black Gauss-Seidel sweep(s) for sigma tau (2I - Lap) u = b; the flow
// steps and reflections.  A warp streams its band top-down as a pipeline of
// S = 1 + 2 sweeps half-sweep stages: at step m it takes row m in (u^k, b),
// runs stage s (red, black, red, ...) on row m-1-s, and finishes row m-S-1
// (flows and reflections from the final u of rows m-S-1 and m-S).  A stage
// reads the row below at the previous stage's version and the row above at
// its own stage's version, whose cells of the other colour -- the only ones
// a half-sweep reads -- are still at the previous stage's version: exactly
// the red-black order.  Each stage needs one more column of halo, so lanes
// 0..SW and 31-SW..31 carry the halo and 2 (32 - 2 (SW + 1)) columns are
// owned per strip.
template <typename S, bool ANISO, int SW>
__global__ void __launch_bounds__(kStripWarps * 32)
    k_binary_dr_strip(BinProblem P, BinState<S> s0, BinState<S> s1, DrCoef D, int R,
                      int nstrips, int nitems) {
    constexpr int NS = 1 + 2 * SW;        // half-sweep stages
    constexpr int HL = SW + 1;            // halo lanes on each side
    constexpr int OUT = 2 * (32 - 2 * HL);  // owned columns per strip
    using PS = Pair<S>;
    using PF = Pair<float>;
    const int lane = threadIdx.x & 31;
    const Grid G = P.g;
    const unsigned full = 0xffffffffu;

    for (int item = blockIdx.x * kStripWarps + (threadIdx.x >> 5); item < nitems;
         item += gridDim.x * kStripWarps) {
        const int x0 = (item % nstrips) * OUT;
        const int r0 = (item / nstrips) * R;
        const int r1 = min(r0 + R, G.H);
        const int c = x0 - 2 * HL + 2 * lane;  // even column of the pair (W is even)
        const bool colin = c >= 0 && c < G.W;
        const bool own = colin && lane >= HL && lane <= 31 - HL;
        const float mxo = c + 1 < G.W - 1 ? 1.f : 0.f;
        // neighbour counts of the two columns in x
        const float ncx_e = (c > 0 ? 1.f : 0.f) + (c < G.W - 1 ? 1.f : 0.f);
        const float ncx_o = 1.f + mxo;
        auto ok_row = [&](int r) { return colin && r >= 0 && r < G.H; };
        // stored pairs stay in their storage type until used: a conversion at
        // the load would wait for the prefetched row at once
        auto ld_s = [&](const S* base, int r) {
            return ok_row(r) ? PS::ld(base + r * G.pitch + c) : PS::zero();
        };
        auto ld_f = [&](const float* base, int r) {
            return ok_row(r) ? PF::ld(base + r * G.pitch + c) : PF::zero();
        };
        auto ld_al = [&](int r) {
            if (!P.alpha.plane) return make_float2(P.alpha.value, P.alpha.value);
            return ld_f(P.alpha.plane, r);
        };
        using SP = typename PS::T;

        float2 V[NS + 2];   // V[k]: u of row m-k (stage k-1 applied; k >= NS: final)
        float2 Bh[NS + 1];  // Bh[k]: b of row m-k
#pragma unroll
        for (int k = 0; k < NS + 2; ++k) V[k] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < NS + 1; ++k) Bh[k] = make_float2(0.f, 0.f);
        SP qby_up = ld_s(s0.qy, r0 - NS - 1);  // qbar_y of the row above the ingested one

        // prefetched inputs of the next ingested row and the next finished row
        const int m_first = r0 - NS, m_last = r1 + NS;
        float2 in_u = ld_f(s0.u, m_first);
        SP in_qx = ld_s(s0.qx, m_first), in_qy = ld_s(s0.qy, m_first);
        SP in_ps = ld_s(s0.ps, m_first), in_pt = ld_s(s0.pt, m_first);
        const int t_first = m_first - NS - 1;
        SP f_qx = ld_s(s0.qx, t_first), f_qy = ld_s(s0.qy, t_first);
        SP f_ps = ld_s(s0.ps, t_first), f_pt = ld_s(s0.pt, t_first);
        float2 f_cs = ld_f(P.Cs, t_first), f_ct = ld_f(P.Ct, t_first), f_al = ld_al(t_first);

#pragma unroll 1
        for (int m = m_first; m <= m_last; ++m) {
            // shift the pipeline: row m enters
#pragma unroll
            for (int k = NS + 1; k > 0; --k) V[k] = V[k - 1];
#pragma unroll
            for (int k = NS; k > 0; --k) Bh[k] = Bh[k - 1];
            // b of row m (zero outside the grid)
            {
                const float2 qx = PS::f2(in_qx), qy = PS::f2(in_qy), qu = PS::f2(qby_up);
                const float2 ps = PS::f2(in_ps), pt = PS::f2(in_pt);
                const float qxl = __shfl_up_sync(full, qx.y, 1);
                const float wy = m < G.H - 1 ? 1.f : 0.f;
                float2 b;
                b.x = -D.sigma * (qx.x - qxl + wy * qy.x - qu.x + pt.x - ps.x);
                b.y = -D.sigma * (mxo * qx.y - qx.x + wy * qy.y - qu.y + pt.y - ps.y);
                const bool ok = ok_row(m);
                Bh[0] = ok ? b : make_float2(0.f, 0.f);
                V[0] = in_u;  // zero outside the grid
                qby_up = in_qy;
            }
            if (m < m_last) {  // next ingested row
                const int r = m + 1;
                in_u = ld_f(s0.u, r);
                in_qx = ld_s(s0.qx, r);
                in_qy = ld_s(s0.qy, r);
                in_ps = ld_s(s0.ps, r);
                in_pt = ld_s(s0.pt, r);
            }
            // half-sweep stages on rows m-1 .. m-NS
#pragma unroll
            for (int st = 0; st < NS; ++st) {
                // j, and so the colour, is the same for the whole warp: one
                // branch, one shuffle per stage
                const int j = m - 1 - st;
                if (j < 0 || j >= G.H) continue;
                const bool red = (st & 1) == 0;          // red: (row + col) even
                const bool act_e = ((j & 1) == 0) == red;  // the pair's even column is active
                const float2 cur = V[st + 1], up = V[st + 2], dn = V[st];
                const float ncy = (j > 0 ? 1.f : 0.f) + (j < G.H - 1 ? 1.f : 0.f);
                const float2 bj = Bh[st + 1];
                if (act_e) {
                    const float left = __shfl_up_sync(full, cur.y, 1);  // u(j, c-1)
                    const float v = __fdividef(bj.x * D.inv_st + (left + cur.y + up.x + dn.x),
                                               D.kappa + ncx_e + ncy);
                    if (colin) V[st + 1].x = v;
                } else {
                    const float right = __shfl_down_sync(full, cur.x, 1);  // u(j, c+2)
                    const float v = __fdividef(bj.y * D.inv_st + (cur.x + right + up.y + dn.y),
                                               D.kappa + ncx_o + ncy);
                    if (colin) V[st + 1].y = v;
                }
            }
            // finish row t = m - NS - 1: flows, reflections, outputs
            const int t = m - NS - 1;
            const float2 uc = V[NS + 1], ud = V[NS];
            const float u_right = __shfl_down_sync(full, uc.x, 1);
            if (t >= r0 && t < r1 && own) {
                const float wy = t < G.H - 1 ? 1.f : 0.f;
                const float gx_e = uc.y - uc.x, gx_o = mxo * (u_right - uc.y);
                const float gy_e = wy * (ud.x - uc.x), gy_o = wy * (ud.y - uc.y);
                float qx_e, qy_e, ps_e, pt_e, qx_o, qy_o, ps_o, pt_o;
                const float2 fqx = PS::f2(f_qx), fqy = PS::f2(f_qy);
                const float2 fps = PS::f2(f_ps), fpt = PS::f2(f_pt);
                binary_dr_flows<S, ANISO>(D, uc.x, gx_e, gy_e, fqx.x, fqy.x, fps.x, fpt.x,
                                          f_al.x, f_cs.x, f_ct.x, qx_e, qy_e, ps_e, pt_e);
                binary_dr_flows<S, ANISO>(D, uc.y, gx_o, gy_o, fqx.y, fqy.y, fps.y, fpt.y,
                                          f_al.y, f_cs.y, f_ct.y, qx_o, qy_o, ps_o, pt_o);
                const int o = t * G.pitch + c;
                PF::st(s1.u + o, uc.x, uc.y);
                PS::st(s1.qx + o, qx_e, qx_o);
                PS::st(s1.qy + o, qy_e, qy_o);
                PS::st(s1.ps + o, ps_e, ps_o);
                PS::st(s1.pt + o, pt_e, pt_o);
            }
            if (m < m_last) {  // inputs of the next finished row
                const int r = t + 1;
                f_qx = ld_s(s0.qx, r);
                f_qy = ld_s(s0.qy, r);
                f_ps = ld_s(s0.ps, r);
                f_pt = ld_s(s0.pt, r);
                f_cs = ld_f(P.Cs, r);
                f_ct = ld_f(P.Ct, r);
                f_al = ld_al(r);
            }
        }
    }
}

// ---- host side -------------------------------------------------------------

bool binary_strip_eligible(const Grid& G, int storage, const float* Cs, const float* Ct,
                           const float* alpha, const BinStateV& a, const BinStateV& b) {
    if (G.W % 2 || G.pitch % 2) return false;
    if ((size_t)G.H * (size_t)G.pitch > (size_t)INT_MAX) return false;
    const size_t es2 = 2 * dtype_size(storage);
    auto al = [](const void* p, size_t n) { return ((uintptr_t)p % n) == 0; };
    if (!al(Cs, 8) || !al(Ct, 8) || (alpha && !al(alpha, 8))) return false;
    for (const BinStateV* s : {&a, &b})
        if (!al(s->u, 8) || !al(s->qx, es2) || !al(s->qy, es2) || !al(s->ps, es2) ||
            !al(s->pt, es2))
            return false;
    return true;
}

template <typename S, bool ANISO>
static cudaError_t launch_bin_strip(const BinProblem& P, const BinState<S>& a,
                                    const BinState<S>& b, const AdmmCoef& K, cudaStream_t st) {
    auto kern = k_binary_strip<S, ANISO>;
    static std::atomic<long long> memo[kMaxDevices];  // warps resident per device
    long long resident = 0;
    {
        const cudaError_t e = strip::device_resident_warps(memo, kern, 0, resident);
        if (e != cudaSuccess) return e;
    }
    const Grid& G = P.g;
    const int nstrips = (G.W + kStripOut - 1) / kStripOut;
    const int R = strip::choose_rows(G.H, nstrips, resident, 4, 64, 3);
    const int nitems = nstrips * ((G.H + R - 1) / R);
    const int blocks = (nitems + kStripWarps - 1) / kStripWarps;
    const int grid = blocks < resident / kStripWarps ? blocks : resident / kStripWarps;
    kern<<<grid, kStripWarps * 32, 0, st>>>(P, a, b, K, R, nstrips, nitems);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t bin_strip_s(const BinProblem& P, const BinStateV& a, const BinStateV& b,
                               bool aniso, const AdmmCoef& K, cudaStream_t st) {
    const BinState<S> A = a.as<S>(), B = b.as<S>();
    return aniso ? launch_bin_strip<S, true>(P, A, B, K, st)
                 : launch_bin_strip<S, false>(P, A, B, K, st);
}

cudaError_t binary_strip_step(int storage, const BinProblem& P, const BinStateV& a,
                              const BinStateV& b, bool aniso, const AdmmCoef& K,
                              cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return bin_strip_s<float>(P, a, b, aniso, K, st);
        case CMF_F16: return bin_strip_s<__half>(P, a, b, aniso, K, st);
        default: return bin_strip_s<__nv_bfloat16>(P, a, b, aniso, K, st);
    }
}

template <typename S, bool ANISO, int SW>
static cudaError_t launch_bin_dr_strip(const BinProblem& P, const BinState<S>& a,
                                       const BinState<S>& b, const DrCoef& D, cudaStream_t st) {
    auto kern = k_binary_dr_strip<S, ANISO, SW>;
    static std::atomic<long long> memo[kMaxDevices];  // warps resident per device
    long long resident = 0;
    {
        const cudaError_t e = strip::device_resident_warps(memo, kern, 0, resident);
        if (e != cudaSuccess) return e;
    }
    const Grid& G = P.g;
    constexpr int OUT = 2 * (32 - 2 * (SW + 1));
    const int nstrips = (G.W + OUT - 1) / OUT;
    const int R = strip::choose_rows(G.H, nstrips, resident, 8, 64, 2 * (1 + 2 * SW) + 1);
    const int nitems = nstrips * ((G.H + R - 1) / R);
    const int blocks = (nitems + kStripWarps - 1) / kStripWarps;
    const int grid = blocks < resident / kStripWarps ? blocks : resident / kStripWarps;
    kern<<<grid, kStripWarps * 32, 0, st>>>(P, a, b, D, R, nstrips, nitems);
    return cudaGetLastError();
}

template <typename S, bool ANISO>
static cudaError_t bin_dr_strip_sw(const BinProblem& P, const BinState<S>& A,
                                   const BinState<S>& B, const DrCoef& D, cudaStream_t st) {
    switch (D.sweeps) {
        case 1: return launch_bin_dr_strip<S, ANISO, 1>(P, A, B, D, st);
        case 2: return launch_bin_dr_strip<S, ANISO, 2>(P, A, B, D, st);
        case 3: return launch_bin_dr_strip<S, ANISO, 3>(P, A, B, D, st);
        default: return launch_bin_dr_strip<S, ANISO, 4>(P, A, B, D, st);
    }
}

template <typename S>
static cudaError_t bin_dr_strip_s(const BinProblem& P, const BinStateV& a, const BinStateV& b,
                                  bool aniso, const DrCoef& D, cudaStream_t st) {
    const BinState<S> A = a.as<S>(), B = b.as<S>();
    return aniso ? bin_dr_strip_sw<S, true>(P, A, B, D, st)
                 : bin_dr_strip_sw<S, false>(P, A, B, D, st);
}

cudaError_t binary_dr_strip_step(int storage, const BinProblem& P, const BinStateV& a,
                                 const BinStateV& b, bool aniso, const DrCoef& D,
                                 cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return bin_dr_strip_s<float>(P, a, b, aniso, D, st);
        case CMF_F16: return bin_dr_strip_s<__half>(P, a, b, aniso, D, st);
        default: return bin_dr_strip_s<__nv_bfloat16>(P, a, b, aniso, D, st);
    }
}

}  // namespace cmf

// ---- certificates by warp strips (Eq. seg:chanvese, Eq. two-label-mf) ------
//
// The same strips and bands as the iteration.  Per output pixel, in float32:
// the primal energy at clip(u, 0, 1), the conservation residual of the flows
// y (q for ADMM; q - tau grad u, p_t + tau u, p_s - tau u for rPDRQ) and the
// max-flow value min(C_s, C_t + div P_alpha(y)).  Each row's pair is added to
// per-lane double-float sums (FP64 from the warp sums on); the block's sums go
// to partials[blockIdx.x].  The grid has exactly eval_blocks(H, W) blocks so
// the partial count is the tile kernel's; eval_tail may reduce them.
namespace cmf {

template <typename S, bool ANISO, bool DR>
__global__ void __launch_bounds__(kStripWarps * 32)
    k_binary_eval_strip(BinProblem P, BinState<S> s, float tau, int R, int nstrips, int nitems,
                        double* partials, EvalTail T) {
    using PS = Pair<S>;
    using PF = Pair<float>;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const Grid G = P.g;
    const unsigned full = 0xffffffffu;
    DF accE = {0.f, 0.f}, accD = {0.f, 0.f}, accR = {0.f, 0.f};

    for (int item = blockIdx.x * kStripWarps + wib; item < nitems;
         item += gridDim.x * kStripWarps) {
        const int cs0 = (item % nstrips) * kStripOut;
        const int r0 = (item / nstrips) * R;
        const int r1 = min(r0 + R, G.H);
        const int c = cs0 - 2 + 2 * lane;
        const bool colin = c >= 0 && c < G.W;
        const bool own = colin && lane >= 1 && lane <= 30;
        const float mxo = c + 1 < G.W - 1 ? 1.f : 0.f;
        auto ok_row = [&](int r) { return colin && r >= 0 && r < G.H; };
        // stored pairs stay in their storage type until used
        auto ld_raw = [&](const S* base, int r) {
            return ok_row(r) ? PS::ld(base + r * G.pitch + c) : PS::zero();
        };
        auto ld_f = [&](const float* base, int r) {
            return ok_row(r) ? PF::ld(base + r * G.pitch + c) : PF::zero();
        };
        auto ld_al = [&](int r) {
            if (!P.alpha.plane) return make_float2(P.alpha.value, P.alpha.value);
            return ld_f(P.alpha.plane, r);
        };
        auto row_w = [&](int r) { return r < G.H - 1 ? 1.f : 0.f; };
        // the inputs of one row, loaded a row ahead of their use
        struct RowIn {
            typename PS::T qx, qy, ps, pt;
            float2 cs, ct, al;
        };
        auto row_in = [&](int r) {
            RowIn x;
            x.qx = ld_raw(s.qx, r);
            x.qy = ld_raw(s.qy, r);
            x.ps = ld_raw(s.ps, r);
            x.pt = ld_raw(s.pt, r);
            x.cs = ld_f(P.Cs, r);
            x.ct = ld_f(P.Ct, r);
            x.al = ld_al(r);
            return x;
        };
        // flows y of row r (zero outside the grid) from q and, for rPDRQ, u of
        // rows r and r+1; every lane takes part in the shuffle
        auto flows = [&](const RowIn& x, int r, float2 u_r, float2 u_d, float2& f_x,
                         float2& f_y) {
            const float2 qx = PS::f2(x.qx), qy = PS::f2(x.qy);
            const float u_right = __shfl_down_sync(full, u_r.x, 1);  // u(r, c+2)
            f_x = qx;
            f_y = qy;
            if (DR) {
                const float wy = row_w(r);
                f_x.x -= tau * (u_r.y - u_r.x);
                f_x.y -= tau * mxo * (u_right - u_r.y);
                f_y.x -= tau * wy * (u_d.x - u_r.x);
                f_y.y -= tau * wy * (u_d.y - u_r.y);
            }
            if (!ok_row(r)) f_x = f_y = make_float2(0.f, 0.f);
        };

        // row r0-1: its y flows and their projections enter the divergence at r0
        float2 u_t = ld_f(s.u, r0 - 1), u_n = ld_f(s.u, r0);
        float2 fx, fy;
        const RowIn x0 = row_in(r0 - 1);
        flows(x0, r0 - 1, u_t, u_n, fx, fy);
        float2 fy_up = fy, py_up;
        project_sel<ANISO>(fx.x, fy.x, x0.al.x);
        project_sel<ANISO>(fx.y, fy.y, x0.al.y);
        py_up = fy;
        u_t = u_n;
        RowIn nx = row_in(r0);
        float2 u_nn = ld_f(s.u, r0 + 1);
#pragma unroll 1
        for (int t = r0; t < r1; ++t) {
            // row t's inputs arrived during the previous step; row t+1's and
            // u of row t+2 go in flight now
            const RowIn x = nx;
            u_n = u_nn;
            if (t + 1 < r1) nx = row_in(t + 1);
            if (t + 2 <= r1) u_nn = ld_f(s.u, t + 2);
            const float2 cs = x.cs, ct = x.ct, al = x.al;
            float2 ps = PS::f2(x.ps), pt = PS::f2(x.pt);
            flows(x, t, u_t, u_n, fx, fy);
            const float wy = row_w(t);
            // primal energy at ub = clip(u, 0, 1)
            const float ub_e = fminf(fmaxf(u_t.x, 0.f), 1.f);
            const float ub_o = fminf(fmaxf(u_t.y, 0.f), 1.f);
            const float ub_r = __shfl_down_sync(full, ub_e, 1);
            const float gx_e = ub_o - ub_e, gx_o = mxo * (ub_r - ub_o);
            const float gy_e = wy * (fminf(fmaxf(u_n.x, 0.f), 1.f) - ub_e);
            const float gy_o = wy * (fminf(fmaxf(u_n.y, 0.f), 1.f) - ub_o);
            const float tv_e = ANISO ? fabsf(gx_e) + fabsf(gy_e) : sqrtf(gx_e * gx_e + gy_e * gy_e);
            const float tv_o = ANISO ? fabsf(gx_o) + fabsf(gy_o) : sqrtf(gx_o * gx_o + gy_o * gy_o);
            const float e_e = (1.f - ub_e) * cs.x + ub_e * ct.x + al.x * tv_e;
            const float e_o = (1.f - ub_o) * cs.y + ub_o * ct.y + al.y * tv_o;
            // conservation residual of y
            if (DR) {
                pt.x += tau * u_t.x;
                pt.y += tau * u_t.y;
                ps.x -= tau * u_t.x;
                ps.y -= tau * u_t.y;
            }
            const float fxl = __shfl_up_sync(full, fx.y, 1);
            const float r_e = fx.x - fxl + wy * fy.x - fy_up.x - ps.x + pt.x;
            const float r_o = mxo * fx.y - fx.x + wy * fy.y - fy_up.y - ps.y + pt.y;
            // max-flow value of P_alpha(y)
            float px = fx.x, py = fy.x, qx_ = fx.y, qy_ = fy.y;
            project_sel<ANISO>(px, py, al.x);
            project_sel<ANISO>(qx_, qy_, al.y);
            const float pxl = __shfl_up_sync(full, qx_, 1);
            const float dp_e = px - pxl + wy * py - py_up.x;
            const float dp_o = mxo * qx_ - px + wy * qy_ - py_up.y;
            if (own) {
                df_add(accE, e_e + e_o);
                df_add(accR, r_e * r_e + r_o * r_o);
                df_add(accD, fminf(cs.x, ct.x + dp_e) + fminf(cs.y, ct.y + dp_o));
            }
            fy_up = fy;
            py_up = make_float2(py, qy_);
            u_t = u_n;
        }
    }
    // block sums, fixed order
    __shared__ double red[3][kStripWarps];
    accE = df_warp_sum(accE);
    accD = df_warp_sum(accD);
    accR = df_warp_sum(accR);
    if (lane == 0) {
        red[0][wib] = df_value(accE);
        red[1][wib] = df_value(accD);
        red[2][wib] = df_value(accR);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, cc = 0.0;
        for (int w = 0; w < kStripWarps; ++w) {
            a += red[0][w];
            b += red[1][w];
            cc += red[2][w];
        }
        double* out = partials + 3 * (size_t)blockIdx.x;
        out[0] = a;
        out[1] = b;
        out[2] = cc;
    }
    eval_tail(T, partials, gridDim.x);
}

template <typename S, bool ANISO, bool DR>
static cudaError_t launch_bin_eval_strip(const BinProblem& P, const BinState<S>& s, float tau,
                                         double* partials, cudaStream_t st,
                                         const EvalTail& T) {
    const Grid& G = P.g;
    // the grid is eval_blocks(H, W) blocks (the partial count every
    // certificate path shares); bands sized for the warps actually resident
    const int blocks = eval_blocks(G.H, G.W);
    static std::atomic<long long> memo[kMaxDevices];  // warps resident per device
    const long long resident = strip::resident_warps(memo, k_binary_eval_strip<S, ANISO, DR>);
    const long long slots = resident > 0 ? resident : (long long)blocks * kStripWarps;
    const int nstrips = (G.W + kStripOut - 1) / kStripOut;
    const int R = strip::choose_rows(G.H, nstrips, slots, 4, 64, 2);
    const int nitems = nstrips * ((G.H + R - 1) / R);
    k_binary_eval_strip<S, ANISO, DR>
        <<<blocks, kStripWarps * 32, 0, st>>>(P, s, tau, R, nstrips, nitems, partials, T);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t bin_eval_strip_s(const BinProblem& P, const BinStateV& sv, bool aniso, bool dr,
                                    float tau, double* partials, cudaStream_t st,
                                    const EvalTail& T) {
    const BinState<S> s = sv.as<S>();
    if (dr)
        return aniso ? launch_bin_eval_strip<S, true, true>(P, s, tau, partials, st, T)
                     : launch_bin_eval_strip<S, false, true>(P, s, tau, partials, st, T);
    return aniso ? launch_bin_eval_strip<S, true, false>(P, s, tau, partials, st, T)
                 : launch_bin_eval_strip<S, false, false>(P, s, tau, partials, st, T);
}

cudaError_t binary_eval_strip(int storage, const BinProblem& P, const BinStateV& s, bool aniso,
                              bool dr, float tau, double* partials, cudaStream_t st,
                              const EvalTail& T) {
    switch (storage) {
        case CMF_F32: return bin_eval_strip_s<float>(P, s, aniso, dr, tau, partials, st, T);
        case CMF_F16: return bin_eval_strip_s<__half>(P, s, aniso, dr, tau, partials, st, T);
        default: return bin_eval_strip_s<__nv_bfloat16>(P, s, aniso, dr, tau, partials, st, T);
    }
}

}  // namespace cmf
