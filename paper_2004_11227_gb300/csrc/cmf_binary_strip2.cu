// Binary ADMM, two iterations per launch by warp strips (Eq. rpADMMII, Eq.
// rpADMMI, pADMM-TY Eq. ADMM:Tai_yuan, ALG1 Eq. iteration:pd:seg): temporal
// blocking of the one-iteration warp-strip kernel of cmf_binary_strip.cu.
#include "cmf_kernels.cuh"
#include "cmf_strip.cuh"

namespace cmf {

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

// ---- two ADMM iterations per launch ----------------------------------------
//
// Temporal blocking of k_binary_strip: stage A makes iteration k+1 of row j
// exactly as k_binary_strip does and keeps it in registers, rounded to the
// storage type as a store and a load would; stage B makes iteration k+2 of
// row j-1 from A's rows j-1 and j.  A is valid on lanes 1..30 (its column
// neighbours come by shuffles), B on lanes 2..29, so a strip advances 56
// columns (cs-4 .. cs+59 covered).  A band of R output rows reads rows
// r0-3 .. r1+1 of iteration k and writes rows r0 .. r1-1 of iteration k+2;
// iteration k+1 never reaches memory.  One launch gives the state two
// launches of k_binary_strip give.
//
// CERT: the launch also computes the certificates of the state it writes
// (primal energy E at clip(u, 0, 1), dual value D of the re-projected flows,
// squared conservation residual; the definitions of the certificate kernels)
// and reduces them with eval_tail, so a check costs no separate pass.  The
// TV term of a pixel needs u at the next column and the next row: lanes
// 2..28 are owned (lane 29 supplies the next column; 54 columns per strip)
// and stage B also makes row r1 (not stored; its u completes the TV terms of
// row r1 - 1, which are added one row late).  Per-pixel terms are summed in
// double-float per lane, one partial triple per block.
constexpr int kStrip2Out = 56;
constexpr int kStrip2OutCert = 54;
constexpr int kCertMaxBlocks = 2048;  // partial triples the workspace holds

template <typename S, bool ANISO, bool CERT>
__global__ void __launch_bounds__(kStripWarps * 32, 4)
    k_binary_strip2(BinProblem P, BinState<S> s0, BinState<S> s1, AdmmCoef K, int R,
                    int nstrips, int nitems, double* partials, EvalTail T) {
    using St = Store<S>;
    using PS = Pair<S>;
    using PF = Pair<float>;
    constexpr int OUT = CERT ? kStrip2OutCert : kStrip2Out;
    const int lane = threadIdx.x & 31;
    const Grid G = P.g;
    const unsigned full = 0xffffffffu;
    DF accE = {0.f, 0.f}, accD = {0.f, 0.f}, accR = {0.f, 0.f};

    for (int item = blockIdx.x * kStripWarps + (threadIdx.x >> 5); item < nitems;
         item += gridDim.x * kStripWarps) {
        const int cs = (item % nstrips) * OUT;
        const int r0 = (item / nstrips) * R;
        const int r1 = min(r0 + R, G.H);
        const int c = cs - 4 + 2 * lane;  // even column of the pair (W is even)
        const bool colin = c >= 0 && c < G.W;
        const bool own = colin && lane >= 2 && lane <= (CERT ? 28 : 29);
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
        // One ADMM step at row t from the row's state x, g at rows t and t+1,
        // the new q_y of the row above and the row's alpha, C_s, C_t: the new
        // state of the row, zero outside the grid.  full_row = false: flows only.
        auto step = [&](const BinRow<S>& x, float2 g_t, float2 g_n, float2& qyn_up, float2 al,
                        float2 csr, float2 ctr, int t, bool full_row, BinRow<S>& y,
                        float2& d_out) {
            const float g_r = __shfl_down_sync(full, g_t.x, 1);  // g(t, c+2)
            const float my = row_w(t) * K.inv_a;
            const float2 qx = PS::f2(x.qx), qy = PS::f2(x.qy);
            float tx_e = qx.x + (g_t.y - g_t.x) * K.inv_a;
            float tx_o = qx.y + (g_r - g_t.y) * (mxo * K.inv_a);
            float ty_e = qy.x + (g_n.x - g_t.x) * my;
            float ty_o = qy.y + (g_n.y - g_t.y) * my;
            project_sel<ANISO>(tx_e, ty_e, al.x);
            project_sel<ANISO>(tx_o, ty_o, al.y);
            const bool in = colin && t >= 0 && t < G.H;
            tx_e = in ? St::rt(tx_e) : 0.f;
            tx_o = in ? St::rt(tx_o) : 0.f;
            ty_e = in ? St::rt(ty_e) : 0.f;
            ty_o = in ? St::rt(ty_o) : 0.f;
            y.qx = PS::pk(tx_e, tx_o);
            y.qy = PS::pk(ty_e, ty_o);
            if (full_row) {
                const float txl = __shfl_up_sync(full, tx_o, 1);  // new q_x at c-1
                const float wy = row_w(t);
                const float d_e = tx_e - txl + wy * ty_e - qyn_up.x;
                const float d_o = mxo * tx_o - tx_e + wy * ty_o - qyn_up.y;
                d_out = make_float2(d_e, d_o);
                const float2 ps = PS::f2(x.ps), pt = PS::f2(x.pt);
                float ps_e, pt_e, u_e, ps_o, pt_o, u_o;
                binary_pu<S>(K, g_t.x, d_e, ps.x, pt.x, x.u.x, csr.x, ctr.x, ps_e, pt_e, u_e);
                binary_pu<S>(K, g_t.y, d_o, ps.y, pt.y, x.u.y, csr.y, ctr.y, ps_o, pt_o, u_o);
                y.ps = in ? PS::pk(ps_e, ps_o) : PS::zero();
                y.pt = in ? PS::pk(pt_e, pt_o) : PS::zero();
                y.u = in ? make_float2(u_e, u_o) : PF::zero();
            } else {
                y.ps = PS::zero();
                y.pt = PS::zero();
                y.u = PF::zero();
                d_out = PF::zero();
            }
            qyn_up = make_float2(ty_e, ty_o);
        };

        // stage A: iteration k+1 of rows r0-2 .. rl (flows only at r0-2)
        // stage B: iteration k+2 of rows r0-1 .. rl-1 (flows only at r0-1);
        // rl = r1, or r1 + 1 with the certificates
        const int rl = r1 + (CERT ? 1 : 0);
        BinRow<S> a, b, nx;
        const int ra = r0 - 2;
        const float2 qy_m3 = PS::f2(ok_row(ra - 1) ? PS::ld(s0.qy + (ra - 1) * G.pitch + c)
                                                   : PS::zero());
        row(ra, a);
        row(ra + 1, b);
        float2 g_t = g_of(a, qy_m3, ra);
        float2 qyn_up = make_float2(0.f, 0.f);
        float2 al_t = ld_al(ra), cs_t = PF::zero(), ct_t = PF::zero();
        BinRow<S> bp;             // A's row j-1
        float2 gb_t = PF::zero();  // g of iteration k+1 at row j-1
        float2 qybn_up = make_float2(0.f, 0.f);
        float2 al_b = PF::zero(), cs_b = PF::zero(), ct_b = PF::zero();
        // certificates: B's previous row (clip(u), its x differences, alpha,
        // whether its TV term is this lane's) and its re-projected new q_y
        float2 ub_p = PF::zero(), gx_p = PF::zero(), al_p = PF::zero();
        float wy_p = 0.f;
        bool tv_p = false;
        float2 py_up = PF::zero();
#pragma unroll 1
        for (int j = ra; j <= rl; ++j) {
            if (j + 2 <= rl + 1) row(j + 2, nx);  // in flight during this row
            float2 al_n = al_t, cs_n = cs_t, ct_n = ct_t;
            if (j + 1 <= rl) {
                al_n = ld_al(j + 1);
                cs_n = ld_f(P.Cs, j + 1);
                ct_n = ld_f(P.Ct, j + 1);
            }
            const float2 g_n = g_of(b, PS::f2(a.qy), j + 1);
            BinRow<S> y;
            float2 d_a;
            step(a, g_t, g_n, qyn_up, al_t, cs_t, ct_t, j, j >= r0 - 1, y, d_a);
            if (j >= r0 - 1) {
                const float2 gb_n = g_of(y, PS::f2(bp.qy), j);  // g of k+1 at row j
                if (j >= r0) {
                    const int t = j - 1;
                    BinRow<S> z;
                    float2 d_b;
                    step(bp, gb_t, gb_n, qybn_up, al_b, cs_b, ct_b, t, t >= r0, z, d_b);
                    const bool mine = own && t >= r0 && t < r1;
                    if (mine) {
                        const int o = t * G.pitch + c;
                        const float2 qx = PS::f2(z.qx), qy = PS::f2(z.qy);
                        const float2 ps = PS::f2(z.ps), pt = PS::f2(z.pt);
                        PS::st(s1.qx + o, qx.x, qx.y);
                        PS::st(s1.qy + o, qy.x, qy.y);
                        PS::st(s1.ps + o, ps.x, ps.y);
                        PS::st(s1.pt + o, pt.x, pt.y);
                        PF::st(s1.u + o, z.u.x, z.u.y);
                    }
                    if (CERT) {
                        const float2 qx = PS::f2(z.qx), qy = PS::f2(z.qy);
                        const float2 ps = PS::f2(z.ps), pt = PS::f2(z.pt);
                        const float wy = row_w(t);
                        const float ub_e = fminf(fmaxf(z.u.x, 0.f), 1.f);
                        const float ub_o = fminf(fmaxf(z.u.y, 0.f), 1.f);
                        const float ub_r = __shfl_down_sync(full, ub_e, 1);  // u(t, c+2)
                        // the previous row's TV term: its vertical difference ends here
                        if (tv_p) {
                            const float gy_e = wy_p * (ub_e - ub_p.x);
                            const float gy_o = wy_p * (ub_o - ub_p.y);
                            const float tv_e = ANISO ? fabsf(gx_p.x) + fabsf(gy_e)
                                                     : sqrtf(gx_p.x * gx_p.x + gy_e * gy_e);
                            const float tv_o = ANISO ? fabsf(gx_p.y) + fabsf(gy_o)
                                                     : sqrtf(gx_p.y * gx_p.y + gy_o * gy_o);
                            df_add(accE, al_p.x * tv_e + al_p.y * tv_o);
                        }
                        // dual value of P_alpha(q), as the certificate kernels take it
                        float px_e = qx.x, py_e = qy.x, px_o = qx.y, py_o = qy.y;
                        project_sel<ANISO>(px_e, py_e, al_b.x);
                        project_sel<ANISO>(px_o, py_o, al_b.y);
                        const float pxl = __shfl_up_sync(full, px_o, 1);
                        if (mine) {
                            df_add(accE, (1.f - ub_e) * cs_b.x + ub_e * ct_b.x +
                                             ((1.f - ub_o) * cs_b.y + ub_o * ct_b.y));
                            const float r_e = d_b.x - ps.x + pt.x, r_o = d_b.y - ps.y + pt.y;
                            df_add(accR, r_e * r_e + r_o * r_o);
                            const float dp_e = px_e - pxl + wy * py_e - py_up.x;
                            const float dp_o = mxo * px_o - px_e + wy * py_o - py_up.y;
                            df_add(accD, fminf(cs_b.x, ct_b.x + dp_e) +
                                             fminf(cs_b.y, ct_b.y + dp_o));
                        }
                        ub_p = make_float2(ub_e, ub_o);
                        gx_p = make_float2(ub_o - ub_e, mxo * (ub_r - ub_o));
                        al_p = al_b;
                        wy_p = wy;
                        tv_p = mine;
                        py_up = make_float2(py_e, py_o);
                    }
                }
                gb_t = gb_n;
            }
            bp = y;
            al_b = al_t;
            cs_b = cs_t;
            ct_b = ct_t;
            a = b;
            b = nx;
            g_t = g_n;
            al_t = al_n;
            cs_t = cs_n;
            ct_t = ct_n;
        }
    }
    if (CERT) {
        block_reduce3_store_df(accE, accD, accR, partials + 3 * (size_t)blockIdx.x);
        eval_tail(T, partials, gridDim.x);
    }
}

// ---- host side -------------------------------------------------------------

template <typename S, bool ANISO, bool CERT>
static cudaError_t launch_bin_strip2(const BinProblem& P, const BinState<S>& a,
                                     const BinState<S>& b, const AdmmCoef& K, double* partials,
                                     const EvalTail& T, cudaStream_t st) {
    auto kern = k_binary_strip2<S, ANISO, CERT>;
    static std::atomic<long long> memo[kMaxDevices];  // warps resident per device
    long long resident = 0;
    {
        const cudaError_t e = strip::device_resident_warps(memo, kern, 0, resident);
        if (e != cudaSuccess) return e;
    }
    const Grid& G = P.g;
    constexpr int OUT = CERT ? kStrip2OutCert : kStrip2Out;
    const int nstrips = (G.W + OUT - 1) / OUT;
    // a band of R rows costs R + 3 steps of stage A and R + 1 of stage B
    const int R = strip::choose_rows(G.H, nstrips, resident, 4, 64, CERT ? 3 : 2);
    const int nitems = nstrips * ((G.H + R - 1) / R);
    const int blocks = (nitems + kStripWarps - 1) / kStripWarps;
    int grid = blocks < resident / kStripWarps ? blocks : resident / kStripWarps;
    if (CERT && grid > kCertMaxBlocks) grid = kCertMaxBlocks;
    kern<<<grid, kStripWarps * 32, 0, st>>>(P, a, b, K, R, nstrips, nitems, partials, T);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t bin_strip2_s(const BinProblem& P, const BinStateV& a, const BinStateV& b,
                                bool aniso, const AdmmCoef& K, double* partials,
                                const EvalTail* cert, cudaStream_t st) {
    const BinState<S> A = a.as<S>(), B = b.as<S>();
    if (cert)
        return aniso ? launch_bin_strip2<S, true, true>(P, A, B, K, partials, *cert, st)
                     : launch_bin_strip2<S, false, true>(P, A, B, K, partials, *cert, st);
    const EvalTail none;
    return aniso ? launch_bin_strip2<S, true, false>(P, A, B, K, nullptr, none, st)
                 : launch_bin_strip2<S, false, false>(P, A, B, K, nullptr, none, st);
}

cudaError_t binary_strip2_step(int storage, const BinProblem& P, const BinStateV& a,
                               const BinStateV& b, bool aniso, const AdmmCoef& K,
                               cudaStream_t st, const EvalTail* cert, double* partials) {
    switch (storage) {
        case CMF_F32: return bin_strip2_s<float>(P, a, b, aniso, K, partials, cert, st);
        case CMF_F16: return bin_strip2_s<__half>(P, a, b, aniso, K, partials, cert, st);
        default: return bin_strip2_s<__nv_bfloat16>(P, a, b, aniso, K, partials, cert, st);
    }
}

int binary_cert_max_blocks() { return kCertMaxBlocks; }

}  // namespace cmf
