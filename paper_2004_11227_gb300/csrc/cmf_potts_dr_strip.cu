// Potts rPDRQ iteration by warp strips (Eq. pdrq:4labels, general L): the
// pipelined red-black Gauss-Seidel preconditioner of Sec. 3 streamed down a
// band of rows, with the labels of one band shared out among the warps of a
// block.
//
// Work unit: one block, a strip of 64 columns (two adjacent columns per lane;
// SW+1 halo lanes on each side) and a band of R output rows.  Phase 1: U =
// sum_j u_j^k for the band's rows and the pipeline's halo rows goes to shared
// memory (one float2 per lane and row, shared by every warp of the block):
// read from the plane the previous launch wrote, or summed from the u_j
// planes on a call's first launch.  Phase 2: warp w runs labels w, w+nw,
// ... down the band: per label, b_i = -sigma (div qbar_i + pbar_i - pbar_s)
// + sigma tau (L u_i - U), 1 + 2 SW half-sweep stages for
// sigma tau ((L+1) I - Lap), then the flow steps and reflections of q_i and
// p_i, written to the output set.  Phase 3 (after a block barrier): the new
// u_i of the band are read back (from L2, written moments before) and summed
// in label order (the next launch's U, written to a plane), and pbar_s is
// reflected.  One shared U per band, instead of one per warp, lets the band be
// several times taller for the same shared memory, so the 2 (1 + 2 SW) + 1
// halo rows every band recomputes weigh less.
#include "cmf_kernels.cuh"
#include "cmf_strip.cuh"

namespace cmf {

using strip::Pair;
using strip::project_sel;

namespace {

constexpr int kDrMaxWarps = 8;  // warps per block at most (one per label group)
constexpr int kDrRmax = 128;    // band rows at most: (128 + 19) x 256 B of U < 48 KB

// The bound of three 8-warp blocks per SM holds a thread to 80 registers (a
// few bytes of spill for one sweep): 24 resident warps for 4-warp blocks
// where 96 registers gave 20 (measured 7% faster; a 64-register bound spilled
// more and ran 20% slower).
template <typename S, bool ANISO, int SW>
__global__ void __launch_bounds__(kDrMaxWarps * 32, 3)
    k_potts_dr_strip(PottsProblem P, PottsState<S> s0, PottsState<S> s1, DrCoef D,
                     const float* __restrict__ U_in, float* __restrict__ U_out, int R,
                     int nstrips, int nitems) {
    constexpr int NS = 1 + 2 * SW;  // half-sweep stages
    constexpr int HL = SW + 1;      // halo lanes on each side
    constexpr int OUT = 2 * (32 - 2 * HL);
    using PS = Pair<S>;
    using PF = Pair<float>;
    extern __shared__ float2 Us[];  // U of rows r0-NS .. r1+NS, one float2 per lane
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const Grid G = P.g;
    const int L = P.L;
    const float stL = D.sigma * D.tau * (float)L, st_ = D.sigma * D.tau;
    const unsigned full = 0xffffffffu;

    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int x0 = (item % nstrips) * OUT;
        const int r0 = (item / nstrips) * R;
        const int r1 = min(r0 + R, G.H);
        const int c = x0 - 2 * HL + 2 * lane;
        const bool colin = c >= 0 && c < G.W;
        const bool own = colin && lane >= HL && lane <= 31 - HL;
        const float mxo = c + 1 < G.W - 1 ? 1.f : 0.f;
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
        const int m_first = r0 - NS, m_last = r1 + NS;

        // phase 1: U = sum_j u_j^k on rows m_first .. m_last, rows shared out
        // (the stored plane holds the same sums, taken in the same order)
        for (int r = m_first + wib; r <= m_last; r += nw) {
            float2 a = make_float2(0.f, 0.f);
            if (ok_row(r)) {
                if (U_in) {
                    a = PF::ld(U_in + r * G.pitch + c);
                } else {
                    const float* ub = s0.u + r * G.pitch + c;
                    for (int l = 0; l < L; ++l) {
                        const float2 v = PF::ld(ub + (size_t)l * G.plane);
                        a.x += v.x;
                        a.y += v.y;
                    }
                }
            }
            Us[(r - m_first) * 32 + lane] = a;
        }
        __syncthreads();

        // phase 2: warp w runs labels w, w + nw, ... through the pipeline
        for (int l = wib; l < L; l += nw) {
            const size_t lo = (size_t)l * G.plane;
            const float* u0 = s0.u + lo;
            const S* qx0 = s0.qx + lo;
            const S* qy0 = s0.qy + lo;
            const S* p0 = s0.p + lo;
            float2 V[NS + 2];   // u of rows m .. m-NS-1, each at its stage's version
            float2 Bh[NS + 1];  // b of rows m .. m-NS
#pragma unroll
            for (int k = 0; k < NS + 2; ++k) V[k] = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < NS + 1; ++k) Bh[k] = make_float2(0.f, 0.f);
            typename PS::T qby_up = ld_s(qy0, m_first - 1);
            float2 in_u = ld_f(u0, m_first);
            typename PS::T in_qx = ld_s(qx0, m_first), in_qy = ld_s(qy0, m_first),
                           in_p = ld_s(p0, m_first);
            float2 in_ps = ld_f(s0.ps, m_first);
            const int t_first = m_first - NS - 1;
            typename PS::T f_qx = ld_s(qx0, t_first), f_qy = ld_s(qy0, t_first);
            // costs of label l: its plane, or (I - c_l)^2 from the image plane
            const float* Cb = P.lev ? P.C : P.C + lo;
            const float lev_l = P.lev ? __ldg(P.lev + l) : 0.f;
            auto ld_cost = [&](int r) {
                if (P.C16)
                    return ok_row(r) ? Pair<__half>::f2(Pair<__half>::ld(P.C16 + lo + r * G.pitch + c))
                                     : PF::zero();
                float2 v = ld_f(Cb, r);
                if (P.lev && ok_row(r)) {
                    v.x = (v.x - lev_l) * (v.x - lev_l);
                    v.y = (v.y - lev_l) * (v.y - lev_l);
                }
                return v;
            };
            typename PS::T f_p = ld_s(p0, t_first);
            float2 f_c = ld_cost(t_first), f_al = ld_al(t_first);
#pragma unroll 1
            for (int m = m_first; m <= m_last; ++m) {
#pragma unroll
                for (int k = NS + 1; k > 0; --k) V[k] = V[k - 1];
#pragma unroll
                for (int k = NS; k > 0; --k) Bh[k] = Bh[k - 1];
                {  // row m enters: u^k and b
                    const float2 qx = PS::f2(in_qx), qy = PS::f2(in_qy), pp = PS::f2(in_p);
                    const float2 qu = PS::f2(qby_up);
                    const float qxl = __shfl_up_sync(full, qx.y, 1);
                    const float wy = m < G.H - 1 ? 1.f : 0.f;
                    const float2 U = Us[(m - m_first) * 32 + lane];
                    float2 b;
                    b.x = -D.sigma * (qx.x - qxl + wy * qy.x - qu.x + pp.x - in_ps.x) +
                          (stL * in_u.x - st_ * U.x);
                    b.y = -D.sigma * (mxo * qx.y - qx.x + wy * qy.y - qu.y + pp.y - in_ps.y) +
                          (stL * in_u.y - st_ * U.y);
                    Bh[0] = ok_row(m) ? b : make_float2(0.f, 0.f);
                    V[0] = in_u;
                    qby_up = in_qy;
                }
                if (m < m_last) {
                    const int r = m + 1;
                    in_u = ld_f(u0, r);
                    in_qx = ld_s(qx0, r);
                    in_qy = ld_s(qy0, r);
                    in_p = ld_s(p0, r);
                    in_ps = ld_f(s0.ps, r);
                }
                // half-sweep stages on rows m-1 .. m-NS; j, and so the
                // colour, is the same for the whole warp: one branch, one
                // shuffle per stage
#pragma unroll
                for (int st = 0; st < NS; ++st) {
                    const int j = m - 1 - st;
                    if (j < 0 || j >= G.H) continue;
                    const bool red = (st & 1) == 0;
                    const bool act_e = ((j & 1) == 0) == red;
                    const float2 cur = V[st + 1], up = V[st + 2], dn = V[st];
                    const float ncy = (j > 0 ? 1.f : 0.f) + (j < G.H - 1 ? 1.f : 0.f);
                    const float2 bj = Bh[st + 1];
                    if (act_e) {
                        const float left = __shfl_up_sync(full, cur.y, 1);
                        const float v = __fdividef(bj.x * D.inv_st + (left + cur.y + up.x + dn.x),
                                                   D.kappa + ncx_e + ncy);
                        if (colin) V[st + 1].x = v;
                    } else {
                        const float right = __shfl_down_sync(full, cur.x, 1);
                        const float v = __fdividef(bj.y * D.inv_st + (cur.x + right + up.y + dn.y),
                                                   D.kappa + ncx_o + ncy);
                        if (colin) V[st + 1].y = v;
                    }
                }
                // row t = m - NS - 1 is final: flow steps and reflections
                const int t = m - NS - 1;
                const float2 uc = V[NS + 1], ud = V[NS];
                const float u_right = __shfl_down_sync(full, uc.x, 1);
                if (t >= r0 && t < r1 && own) {
                    const float wy = t < G.H - 1 ? 1.f : 0.f;
                    const float gx[2] = {uc.y - uc.x, mxo * (u_right - uc.y)};
                    const float gy[2] = {wy * (ud.x - uc.x), wy * (ud.y - uc.y)};
                    const float2 fqx = PS::f2(f_qx), fqy = PS::f2(f_qy), fp = PS::f2(f_p);
                    const float qbx[2] = {fqx.x, fqx.y}, qby[2] = {fqy.x, fqy.y};
                    const float pb[2] = {fp.x, fp.y}, cc[2] = {f_c.x, f_c.y};
                    const float al[2] = {f_al.x, f_al.y}, u[2] = {uc.x, uc.y};
                    float oqx[2], oqy[2], op[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const float q1 = qbx[e] - D.tau * gx[e], q2 = qby[e] - D.tau * gy[e];
                        float tx = 2.f * q1 - qbx[e], ty = 2.f * q2 - qby[e];
                        project_sel<ANISO>(tx, ty, al[e]);
                        oqx[e] = qbx[e] + D.rho * (tx - q1);
                        oqy[e] = qby[e] + D.rho * (ty - q2);
                        const float p1 = pb[e] + D.tau * u[e];
                        op[e] = pb[e] + D.rho * (fminf(2.f * p1 - pb[e], cc[e]) - p1);
                    }
                    const int o = t * G.pitch + c;
                    PF::st(s1.u + lo + o, uc.x, uc.y);
                    PS::st(s1.qx + lo + o, oqx[0], oqx[1]);
                    PS::st(s1.qy + lo + o, oqy[0], oqy[1]);
                    PS::st(s1.p + lo + o, op[0], op[1]);
                }
                if (m < m_last) {
                    const int r = t + 1;
                    f_qx = ld_s(qx0, r);
                    f_qy = ld_s(qy0, r);
                    f_p = ld_s(p0, r);
                    f_c = ld_cost(r);
                    f_al = ld_al(r);
                }
            }
        }
        // the band's new u_i of every label are written (and visible to the
        // block after the barrier); U may be overwritten by the next item
        __syncthreads();

        // phase 3: pbar_s reflection with the sum of the new u_i, rows shared out
        if (own)
            for (int t = r0 + wib; t < r1; t += nw) {
                const int o = t * G.pitch + c;
                float2 us = make_float2(0.f, 0.f);
                for (int l = 0; l < L; ++l) {
                    // coherent load: written by this block's warps in this launch
                    const float2 v = __ldcg(reinterpret_cast<const float2*>(
                        s1.u + (size_t)l * G.plane + o));
                    us.x += v.x;
                    us.y += v.y;
                }
                if (U_out) PF::st(U_out + o, us.x, us.y);
                const float2 pbs = PF::ld(s0.ps + o);
                const float ps1x = pbs.x - D.tau * us.x, ps1y = pbs.y - D.tau * us.y;
                PF::st(s1.ps + o, pbs.x + D.rho * ((2.f * ps1x - pbs.x + D.tau) - ps1x),
                       pbs.y + D.rho * ((2.f * ps1y - pbs.y + D.tau) - ps1y));
            }
    }
}

}  // namespace

// ---- host side -------------------------------------------------------------

// Warps per block for L labels.  Every warp runs ceil(L / nw) pipelines and
// the block waits for the slowest, so the score is the share of the warps'
// label passes that do work, times the band's sharing (up to four warps);
// ties go to fewer idle passes, then to the count nearest four (at 80
// registers a thread, 21-25 warps stay resident per SM for any count).
static int dr_warps(int L) {
    int best = 1;
    double best_score = 0.0, best_eff = 0.0;
    for (int nw = 1; nw <= kDrMaxWarps; ++nw) {
        const int rounds = (L + nw - 1) / nw;
        const double eff = (double)L / (double)(nw * rounds);
        const double score = eff * (double)(nw < 4 ? nw : 4) / 4.0;
        const bool tie = score > best_score - 1e-12 && score < best_score + 1e-12;
        if (score > best_score + 1e-12 || (tie && eff > best_eff + 1e-12) ||
            (tie && eff > best_eff - 1e-12 && abs(nw - 4) < abs(best - 4))) {
            best_score = score;
            best_eff = eff;
            best = nw;
        }
    }
    return best;
}

template <typename S, bool ANISO, int SW>
static cudaError_t launch_potts_dr_strip(const PottsProblem& P, const PottsState<S>& a,
                                         const PottsState<S>& b, const DrCoef& D,
                                         const float* U_in, float* U_out, cudaStream_t st) {
    constexpr int NS = 1 + 2 * SW;
    constexpr int OUT = 2 * (32 - 2 * (SW + 1));
    auto kern = k_potts_dr_strip<S, ANISO, SW>;
    const int nw = dr_warps(P.L);
    auto dyn_for = [](int r) { return (size_t)(r + 2 * NS + 1) * 32 * sizeof(float2); };
    // blocks resident per device, per warp count (the occupancy query runs
    // once per device and block shape; shared memory sized for the tallest band)
    static std::atomic<long long> memo[kDrMaxWarps + 1][kMaxDevices];
    long long resident = 0;
    {
        const cudaError_t e = per_device(
            memo[nw],
            [&](int dev, long long& v) -> cudaError_t {
                int sms = 0, blocks = 0;
                cudaError_t e2;
                if ((e2 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) !=
                    cudaSuccess)
                    return e2;
                if ((e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                         &blocks, kern, nw * 32, dyn_for(kDrRmax))) != cudaSuccess)
                    return e2;
                v = (long long)sms * (blocks > 0 ? blocks : 1);
                return cudaSuccess;
            },
            resident);
        if (e != cudaSuccess) return e;
    }
    const Grid& G = P.g;
    const int nstrips = (G.W + OUT - 1) / OUT;
    // band height: fewest rounds of blocks, each costing its rows plus halo
    const int R = strip::choose_rows(G.H, nstrips, resident, 8, kDrRmax, 2 * NS + 1);
    const int nitems = nstrips * ((G.H + R - 1) / R);
    const int grid = nitems < resident ? nitems : (int)resident;
    kern<<<grid, nw * 32, dyn_for(R), st>>>(P, a, b, D, U_in, U_out, R, nstrips, nitems);
    return cudaGetLastError();
}

template <typename S, bool ANISO>
static cudaError_t potts_dr_strip_sw(const PottsProblem& P, const PottsState<S>& A,
                                     const PottsState<S>& B, const DrCoef& D, const float* U_in,
                                     float* U_out, cudaStream_t st) {
    switch (D.sweeps) {
        case 1: return launch_potts_dr_strip<S, ANISO, 1>(P, A, B, D, U_in, U_out, st);
        case 2: return launch_potts_dr_strip<S, ANISO, 2>(P, A, B, D, U_in, U_out, st);
        case 3: return launch_potts_dr_strip<S, ANISO, 3>(P, A, B, D, U_in, U_out, st);
        default: return launch_potts_dr_strip<S, ANISO, 4>(P, A, B, D, U_in, U_out, st);
    }
}

template <typename S>
static cudaError_t potts_dr_strip_s(const PottsProblem& P, const PottsStateV& a,
                                    const PottsStateV& b, bool aniso, const DrCoef& D,
                                    const float* U_in, float* U_out, cudaStream_t st) {
    const PottsState<S> A = a.as<S>(), B = b.as<S>();
    return aniso ? potts_dr_strip_sw<S, true>(P, A, B, D, U_in, U_out, st)
                 : potts_dr_strip_sw<S, false>(P, A, B, D, U_in, U_out, st);
}

cudaError_t potts_dr_strip_step(int storage, const PottsProblem& P, const PottsStateV& a,
                                const PottsStateV& b, bool aniso, const DrCoef& D,
                                const float* U_in, float* U_out, cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return potts_dr_strip_s<float>(P, a, b, aniso, D, U_in, U_out, st);
        case CMF_F16: return potts_dr_strip_s<__half>(P, a, b, aniso, D, U_in, U_out, st);
        default: return potts_dr_strip_s<__nv_bfloat16>(P, a, b, aniso, D, U_in, U_out, st);
    }
}

}  // namespace cmf
