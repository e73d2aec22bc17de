// Potts ADMM iteration by warp strips (Eq. multi:fg:4, the Eckstein-Bertsekas
// Potts equations after Thm 2, and pADMM-TY, Eq. mADMM:Tai_yuan).
//
// Work unit: one warp, a strip of 64 columns (two adjacent columns per lane)
// and a band of R output rows.  The warp walks the labels one after another;
// for each label it streams down the band row by row, keeping the stencil's
// rolling values (g of the next row, the previous row's new q_y) in registers
// and exchanging column neighbours with warp shuffles.  There are no block
// barriers and no shared-memory halo tiles; loads of row t+2 are in flight
// while row t is computed.  Lanes cover columns cs-2 .. cs+61 and own the
// output columns cs .. cs+59; lane 0 and lane 31 only carry the halo.
//
// Multiplier representation.  Every ADMM variant updates u_i linearly in
// p_s^{k+1}: u_i^{k+1} = v_i + cu p_s^{k+1}.  This kernel stores
// w_i = v_i instead of u_i^{k+1}, so the labels need no second pass once
// p_s^{k+1} is known, and it reads u_i^k = w_i + cu_in p_s^k (cu_in = 0 when
// the input holds u itself).  k_potts_strip_finalize turns w back into u.
//
// The per-label shares of the p_s update are summed in shared memory (one
// float2 per lane and band row); p_s^{k+1} is formed after the last label.
#include <climits>

#include "cmf_kernels.cuh"
#include "cmf_strip.cuh"

namespace cmf {

using strip::kStripOut;
using strip::kStripWarps;
using strip::Pair;
using strip::project_sel;

namespace {

constexpr int kStripRmax = 24;  // band rows at most (shared accumulators: 24 KB per
                                // block, so seven blocks of 72 registers fit an SM)

// State values of one row of one label at this lane's column pair (p_s is
// float32 whatever the flow storage).
template <typename S>
struct RowVals {
    typename Pair<S>::T qx, qy, p;
    float2 ps, w;
};

}  // namespace

// One work item of the Potts strip kernels: strip `cs` (64 columns, two per
// lane, 60 owned), band rows r0 .. r1-1, all labels.  CS: the cost source
// (kCostF32 planes, kCostLevels, kCostF16 planes), a template parameter so
// each instantiation carries only its own loads.  p_s is float32 whatever the
// flow storage S.  Arguments by value: the caller's copies stay in registers
// or the parameter bank.  ODDW: the grid may have an odd width; the pair of
// its last column is (W-1, W), whose second element falls on the padding
// column.  That element is loaded as it is (whatever the padding holds) and
// never stored; the one value of it that reaches a grid column, g at the
// padding column (through the last column's x-difference, whose weight is
// zero), is selected to zero after it is computed.  Masking the loaded values
// instead would consume each prefetched row as soon as it is loaded (measured:
// twice the time per item).  The single-problem solver takes even widths only
// and compiles without these masks.
template <typename S, bool ANISO, int CS, bool ODDW = false>
__device__ __forceinline__ void potts_strip_item(const PottsProblem P, const PottsState<S> s0,
                                                 const PottsState<S> s1, const AdmmCoef K,
                                                 const float cu_in, const int cs, const int r0,
                                                 const int r1, float2 (*acc)[32],
                                                 const int lane) {
    using St = Store<S>;
    using PS = Pair<S>;
    using PF = Pair<float>;
    using PH = Pair<__half>;
    const Grid G = P.g;
    const int L = P.L;
    const unsigned full = 0xffffffffu;
    const int c = cs - 2 + 2 * lane;  // even column of the pair (W is even)
    const bool colin = c >= 0 && c < G.W;
    const bool own = colin && lane >= 1 && lane <= 30;
    const float mxo = c + 1 < G.W - 1 ? 1.f : 0.f;  // odd column is not the last
    const bool oddin = !ODDW || c + 1 < G.W;        // the pair's second column exists
    const float mxe = (!ODDW || c < G.W - 1) ? 1.f : 0.f;  // even column is not the last
    auto row_ok = [&](int r) { return colin && r >= 0 && r < G.H; };
    // weight of a row's own y term: row H-1 has no forward difference
    auto row_w = [&](int r) { return r < G.H - 1 ? 1.f : 0.f; };

    // one row of state at (r, c..c+1): zero outside the grid
    auto load_row = [&](const S* qx, const S* qy, const S* pp, const float* w, int r,
                        RowVals<S>& x) {
        const bool ok = row_ok(r);
        const int o = r * G.pitch + c;
        x.qx = ok ? PS::ld(qx + o) : PS::zero();
        x.qy = ok ? PS::ld(qy + o) : PS::zero();
        x.p = ok ? PS::ld(pp + o) : PS::zero();
        x.ps = ok ? PF::ld(s0.ps + o) : PF::zero();
        x.w = ok ? PF::ld(w + o) : PF::zero();
    };
    // g = div q + p_i - p_s - u_i / c at row r, given the row above's q_y
    // (outside the grid the loaded values are zero)
    auto g_of = [&](const RowVals<S>& x, float2 qy_up, int r) {
        const float2 qx = PS::f2(x.qx), qy = PS::f2(x.qy), p = PS::f2(x.p);
        const float2 ps = x.ps;
        const float qx_left = __shfl_up_sync(full, qx.y, 1);
        const float wy = row_w(r);
        const float u_e = fmaf(cu_in, ps.x, x.w.x), u_o = fmaf(cu_in, ps.y, x.w.y);
        float2 g;
        g.x = qx.x - qx_left + wy * qy.x - qy_up.x + p.x - ps.x - u_e * K.inv_c;
        g.y = mxo * qx.y - qx.x + wy * qy.y - qy_up.y + p.y - ps.y - u_o * K.inv_c;
        if (ODDW) g.y = oddin ? g.y : 0.f;  // the padding column: finite, weight zero
        return g;
    };

    // q^{k+1} = P_alpha(q + grad g / a) at row t of this pair, from g at
    // rows t and t+1 (zero outside the grid)
    struct QN {
        float tx_e, tx_o, ty_e, ty_o;
    };
    auto q_new = [&](const RowVals<S>& x, float2 g_t, float2 g_b, float2 al, int t) {
        const float g_r = __shfl_down_sync(full, g_t.x, 1);  // g(t, c+2)
        const float my = row_w(t) * K.inv_a;
        const float2 qx = PS::f2(x.qx), qy = PS::f2(x.qy);
        QN q;
        q.tx_e = qx.x + (g_t.y - g_t.x) * (ODDW ? mxe * K.inv_a : K.inv_a);
        q.tx_o = qx.y + (g_r - g_t.y) * (mxo * K.inv_a);
        q.ty_e = qy.x + (g_b.x - g_t.x) * my;
        q.ty_o = qy.y + (g_b.y - g_t.y) * my;
        project_sel<ANISO>(q.tx_e, q.ty_e, al.x);
        project_sel<ANISO>(q.tx_o, q.ty_o, al.y);
        const bool in = colin && t >= 0 && t < G.H;
        q.tx_e = in ? St::rt(q.tx_e) : 0.f;
        q.tx_o = (in && oddin) ? St::rt(q.tx_o) : 0.f;
        q.ty_e = in ? St::rt(q.ty_e) : 0.f;
        q.ty_o = (in && oddin) ? St::rt(q.ty_o) : 0.f;
        return q;
    };

#pragma unroll 1
    for (int l = 0; l < L; ++l) {
        const size_t lo = (size_t)l * G.plane;
        const S* qx0 = s0.qx + lo;
        const S* qy0 = s0.qy + lo;
        const S* p0 = s0.p + lo;
        const float* w0 = s0.u + lo;
        // costs of label l: its plane, or (I - c_l)^2 from the image plane
        const float* Cb = CS == kCostLevels ? P.C : P.C + lo;
        const __half* Ch = CS == kCostF16 ? P.C16 + lo : nullptr;
        const float lev_l = CS == kCostLevels ? __ldg(P.lev + l) : 0.f;
        S* qx1 = s1.qx + lo;
        S* qy1 = s1.qy + lo;
        S* p1o = s1.p + lo;
        float* w1 = s1.u + lo;
        auto row = [&](int r, RowVals<S>& x) { load_row(qx0, qy0, p0, w0, r, x); };
        // costs at row r (zero outside the grid; never used there), a select
        // rather than a branch on the lane's bounds
        auto ld_c = [&](int r) {
            const bool ok = row_ok(r);
            float2 v;
            if (CS == kCostF16)
                v = ok ? PH::f2(PH::ld(Ch + r * G.pitch + c)) : PF::zero();
            else
                v = ok ? PF::ld(Cb + r * G.pitch + c) : PF::zero();
            if (CS == kCostLevels) {
                v.x = (v.x - lev_l) * (v.x - lev_l);
                v.y = (v.y - lev_l) * (v.y - lev_l);
            }
            return v;
        };
        auto ld_al = [&](int r) {
            if (!P.alpha.plane) return make_float2(P.alpha.value, P.alpha.value);
            return row_ok(r) ? PF::ld(P.alpha.plane + r * G.pitch + c) : PF::zero();
        };
        // d = div q^{k+1} at output row t from the new q of rows t and t-1,
        // then p_i^{k+1}, w_i and this label's share of the p_s update
        auto finish = [&](int t, const QN& q, float2 qy_up, const RowVals<S>& x, float2 cl,
                          float2 g) {
            const float txl = __shfl_up_sync(full, q.tx_o, 1);  // new q_x at c-1
            const float wy = row_w(t);
            const float d_e = q.tx_e - txl + wy * q.ty_e - qy_up.x;
            const float d_o = mxo * q.tx_o - q.tx_e + wy * q.ty_o - qy_up.y;
            const float2 pv = PS::f2(x.p), ps = x.ps;
            const float u_e = fmaf(cu_in, ps.x, x.w.x), u_o = fmaf(cu_in, ps.y, x.w.y);
            float sa_e = 0.f, sb_e = 0.f, sa_o = 0.f, sb_o = 0.f, v_e, v_o;
            const float p1_e =
                potts_label_pu<S>(K, g.x, d_e, pv.x, ps.x, u_e, cl.x, sa_e, sb_e, v_e);
            const float p1_o =
                potts_label_pu<S>(K, g.y, d_o, pv.y, ps.y, u_o, cl.y, sa_o, sb_o, v_o);
            float2& ac = acc[t - r0][lane];
            const float2 share = make_float2(sa_e + sb_e, sa_o + sb_o);
            if (l == 0) {
                ac = share;
            } else {
                ac.x += share.x;
                ac.y += share.y;
            }
            if (own) {
                const int o = t * G.pitch + c;
                if (!ODDW || oddin) {
                    PS::st(qx1 + o, q.tx_e, q.tx_o);
                    PS::st(qy1 + o, q.ty_e, q.ty_o);
                    PS::st(p1o + o, p1_e, p1_o);
                    PF::st(w1 + o, v_e, v_o);
                } else {  // the last column alone
                    St::st(qx1 + o, q.tx_e);
                    St::st(qy1 + o, q.ty_e);
                    St::st(p1o + o, p1_e);
                    w1[o] = v_e;
                }
            }
        };

        // top-down: step t makes q^{k+1} of row t and finishes row t;
        // row t+2 is loaded during the step
        RowVals<S> a, b, nx;
        const int rm2 = r0 - 2;
        const float2 qy_m2 =
            PS::f2((colin && rm2 >= 0) ? PS::ld(qy0 + rm2 * G.pitch + c) : PS::zero());
        row(r0 - 1, a);
        row(r0, b);
        float2 g_t = g_of(a, qy_m2, r0 - 1);
        float2 qyn_up = make_float2(0.f, 0.f);  // new q_y of the row above
        float2 al_t = ld_al(r0 - 1), cl_t = PF::zero(), al_n = al_t, cl_n = cl_t;
#pragma unroll 1
        for (int t = r0 - 1; t < r1; ++t) {
            if (t + 2 <= r1) row(t + 2, nx);
            if (t + 1 < r1) {
                al_n = ld_al(t + 1);
                cl_n = ld_c(t + 1);
            }
            const float2 g_n = g_of(b, PS::f2(a.qy), t + 1);
            const QN q = q_new(a, g_t, g_n, al_t, t);
            if (t >= r0) finish(t, q, qyn_up, a, cl_t, g_t);
            qyn_up = make_float2(q.ty_e, q.ty_o);
            a = b;
            b = nx;
            g_t = g_n;
            al_t = al_n;
            cl_t = cl_n;
        }
    }

    // p_s^{k+1} on the band from the summed label shares
#pragma unroll 1
    for (int t = r0; t < r1; ++t) {
        if (!own) continue;
        const int o = t * G.pitch + c;
        const float2 ps = PF::ld(s0.ps + o);
        const float2 ac = acc[t - r0][lane];
        if (!ODDW || oddin)
            PF::st(s1.ps + o, potts_ps_update(K, ps.x, ac.x, 0.f),
                   potts_ps_update(K, ps.y, ac.y, 0.f));
        else
            s1.ps[o] = potts_ps_update(K, ps.x, ac.x, 0.f);
    }
}

// One launch of the single-problem solver: every work item is a strip and a
// band of R rows.
template <typename S, bool ANISO, int CS>
__global__ void __launch_bounds__(kStripWarps * 32, 7)
    k_potts_strip(PottsProblem P, PottsState<S> s0, PottsState<S> s1, AdmmCoef K, float cu_in,
                  int R, int nstrips, int nitems) {
    __shared__ float2 acc_s[kStripWarps][kStripRmax][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float2(*acc)[32] = acc_s[wib];
    for (int item = blockIdx.x * kStripWarps + wib; item < nitems;
         item += gridDim.x * kStripWarps) {
        const int cs = (item % nstrips) * kStripOut;
        const int r0 = (item / nstrips) * R;
        const int r1 = min(r0 + R, P.g.H);
        potts_strip_item<S, ANISO, CS>(P, s0, s1, K, cu_in, cs, r0, r1, acc, lane);
    }
}

// Batched Potts ADMM by warp strips: the strip items of every strip-eligible
// Potts instance of a batch in one table of (instance, item) pairs; a warp
// takes its item's problem, state sets and coefficients from the instance's
// descriptor and skips items of retired instances (per-instance convergence
// mask).  parity 0: caller's buffers -> workspace, 1: back; first: the
// chunk's first iteration reads u itself, later ones the w form.  Three
// blocks per SM: each warp holds its instance's problem and coefficients in
// registers (the single-problem kernel has them in the parameter bank); at
// four the 128-register bound spilled, and the spill reloads sat on the row
// pipeline (measured: 4% slower for even widths, 2x for odd ones).
template <typename S, bool ANISO, bool ODDW>
__global__ void __launch_bounds__(kStripWarps * 32, 3)
    k_batch_potts_strip(const BatchDesc* __restrict__ desc, const int2* __restrict__ items,
                        int nitems, int parity, int first) {
    __shared__ float2 acc_s[kStripWarps][kStripRmax][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float2(*acc)[32] = acc_s[wib];
    for (int it = blockIdx.x * kStripWarps + wib; it < nitems; it += gridDim.x * kStripWarps) {
        const int2 e = items[it];
        const BatchDesc* D = desc + e.x;
        if (!D->active) continue;
        const int nstrips = D->sp_nstrips, R = D->sp_rows;
        const PottsStateV a = parity ? D->pw : D->pu, b = parity ? D->pu : D->pw;
        const PottsProblem P = D->pp;
        const AdmmCoef K = D->ak;
        const int cs = (e.y % nstrips) * kStripOut;
        const int r0 = (e.y / nstrips) * R;
        const int r1 = min(r0 + R, P.g.H);
        potts_strip_item<S, ANISO, kCostF32, ODDW>(P, a.as<S>(), b.as<S>(), K,
                                                   first ? 0.f : K.cu, cs, r0, r1, acc, lane);
    }
}

// u_i = w_i + cu p_s on the owned pixels of every item of an active strip
// instance (the state is in the caller's buffers after an even chunk).
__global__ void k_batch_potts_strip_finalize(const BatchDesc* __restrict__ desc,
                                             const int2* __restrict__ items, int nitems) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int it = blockIdx.x * kStripWarps + wib; it < nitems; it += gridDim.x * kStripWarps) {
        const int2 e = items[it];
        const BatchDesc* D = desc + e.x;
        if (!D->active) continue;
        const Grid G = D->pp.g;
        const int cs = (e.y % D->sp_nstrips) * kStripOut;
        const int r0 = (e.y / D->sp_nstrips) * D->sp_rows;
        const int r1 = min(r0 + D->sp_rows, G.H);
        const int c = cs - 2 + 2 * lane;
        if (lane < 1 || lane > 30 || c >= G.W) continue;
        const float cu = D->ak.cu;
        float* u = D->pu.u;
        const float* ps = D->pu.ps;
        const bool pair = c + 1 < G.W;  // else the last column of an odd width alone
        for (int r = r0; r < r1; ++r) {
            const size_t k = G.idx(r, c);
            if (pair) {
                const float2 s = Pair<float>::ld(ps + k);
                for (int l = 0; l < D->pp.L; ++l) {
                    float2* q = reinterpret_cast<float2*>(u + (size_t)l * G.plane + k);
                    float2 v = *q;
                    v.x += cu * s.x;
                    v.y += cu * s.y;
                    *q = v;
                }
            } else {
                const float s = ps[k];
                for (int l = 0; l < D->pp.L; ++l) u[(size_t)l * G.plane + k] += cu * s;
            }
        }
    }
}

int potts_strip_max_rows() { return kStripRmax; }

template <typename S, bool ANISO, bool ODDW>
static cudaError_t launch_batch_strip(const BatchDesc* desc, const int2* items, int nitems,
                                      int parity, int first, cudaStream_t st) {
    auto kern = k_batch_potts_strip<S, ANISO, ODDW>;
    static std::atomic<long long> memo[kMaxDevices];  // warps resident per device
    long long resident = 0;
    {
        const cudaError_t e = strip::device_resident_warps(memo, kern, 0, resident);
        if (e != cudaSuccess) return e;
    }
    const int blocks = (nitems + kStripWarps - 1) / kStripWarps;
    const int grid = blocks < resident / kStripWarps ? blocks : resident / kStripWarps;
    kern<<<grid, kStripWarps * 32, 0, st>>>(desc, items, nitems, parity, first);
    return cudaGetLastError();
}

template <bool ODDW>
static cudaError_t batch_strip_step_o(int storage, bool aniso, const BatchDesc* desc,
                                      const int2* items, int nitems, int parity, int first,
                                      cudaStream_t st) {
    switch (storage) {
        case CMF_F32:
            return aniso ? launch_batch_strip<float, true, ODDW>(desc, items, nitems, parity, first, st)
                         : launch_batch_strip<float, false, ODDW>(desc, items, nitems, parity, first,
                                                                  st);
        case CMF_F16:
            return aniso ? launch_batch_strip<__half, true, ODDW>(desc, items, nitems, parity, first,
                                                                  st)
                         : launch_batch_strip<__half, false, ODDW>(desc, items, nitems, parity,
                                                                   first, st);
        default:
            return aniso ? launch_batch_strip<__nv_bfloat16, true, ODDW>(desc, items, nitems, parity,
                                                                         first, st)
                         : launch_batch_strip<__nv_bfloat16, false, ODDW>(desc, items, nitems,
                                                                          parity, first, st);
    }
}

cudaError_t batch_potts_strip_step(int storage, bool aniso, bool odd_width, const BatchDesc* desc,
                                   const int2* items, int nitems, int parity, int first,
                                   cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    return odd_width
               ? batch_strip_step_o<true>(storage, aniso, desc, items, nitems, parity, first, st)
               : batch_strip_step_o<false>(storage, aniso, desc, items, nitems, parity, first, st);
}

cudaError_t batch_potts_strip_finalize(const BatchDesc* desc, const int2* items, int nitems,
                                       cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const int blocks = (nitems + kStripWarps - 1) / kStripWarps;
    const int grid = blocks < 8 * sms ? blocks : 8 * sms;
    k_batch_potts_strip_finalize<<<grid, kStripWarps * 32, 0, st>>>(desc, items, nitems);
    return cudaGetLastError();
}

// u_i = w_i + cu p_s on every label plane (turns the strip kernel's output
// back into the multipliers themselves).
__global__ void k_potts_strip_finalize(Grid G, int L, float* u, const float* ps, float cu) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (c >= G.W) return;
    const size_t k = G.idx(r, c);
    const float s = cu * __ldg(ps + k);
#pragma unroll 4
    for (int l = 0; l < L; ++l) u[(size_t)l * G.plane + k] += s;
}

// ---- host side -------------------------------------------------------------

bool potts_strip_eligible(const Grid& G, int storage, const float* C, const float* alpha,
                          const PottsStateV& a, const PottsStateV& b, bool odd_width_ok) {
    if ((G.W % 2 && !odd_width_ok) || G.pitch % 2) return false;
    if (G.W % 2 && G.pitch < G.W + 1) return false;  // the last pair reads column W
    if ((size_t)G.H * (size_t)G.pitch > (size_t)INT_MAX) return false;
    const size_t es2 = 2 * dtype_size(storage);
    auto al = [](const void* p, size_t n) { return ((uintptr_t)p % n) == 0; };
    if (!al(C, 8) || (alpha && !al(alpha, 8))) return false;
    for (const PottsStateV* s : {&a, &b})
        if (!al(s->u, 8) || !al(s->qx, es2) || !al(s->qy, es2) || !al(s->p, es2) ||
            !al(s->ps, 8))
            return false;
    return true;
}

template <typename S, bool ANISO, int CS>
static cudaError_t launch_strip(const PottsProblem& P, const PottsState<S>& a,
                                const PottsState<S>& b, const AdmmCoef& K, float cu_in,
                                cudaStream_t st) {
    auto kern = k_potts_strip<S, ANISO, CS>;
    static std::atomic<long long> memo[kMaxDevices];  // warps resident per device
    long long resident = 0;
    {
        const cudaError_t e = strip::device_resident_warps(memo, kern, 0, resident);
        if (e != cudaSuccess) return e;
    }
    const Grid& G = P.g;
    const int nstrips = (G.W + kStripOut - 1) / kStripOut;
    // band height: fewest rounds of work items over the resident warps, each
    // round costing R + 3 rows (the band plus its halo rows)
    const int best_r = strip::choose_rows(G.H, nstrips, resident, 8, kStripRmax, 3);
    const int nitems = nstrips * ((G.H + best_r - 1) / best_r);
    const int blocks = (nitems + kStripWarps - 1) / kStripWarps;
    const int grid = blocks < resident / kStripWarps ? blocks : resident / kStripWarps;
    kern<<<grid, kStripWarps * 32, 0, st>>>(P, a, b, K, cu_in, best_r, nstrips, nitems);
    return cudaGetLastError();
}

template <typename S, int CS>
static cudaError_t strip_step_cs(const PottsProblem& P, const PottsState<S>& A,
                                 const PottsState<S>& B, bool aniso, const AdmmCoef& K,
                                 float cu_in, cudaStream_t st) {
    return aniso ? launch_strip<S, true, CS>(P, A, B, K, cu_in, st)
                 : launch_strip<S, false, CS>(P, A, B, K, cu_in, st);
}

template <typename S>
static cudaError_t strip_step_s(const PottsProblem& P, const PottsStateV& a,
                                const PottsStateV& b, bool aniso, const AdmmCoef& K,
                                float cu_in, cudaStream_t st) {
    const PottsState<S> A = a.as<S>(), B = b.as<S>();
    switch (cost_src(P)) {
        case kCostLevels: return strip_step_cs<S, kCostLevels>(P, A, B, aniso, K, cu_in, st);
        case kCostF16: return strip_step_cs<S, kCostF16>(P, A, B, aniso, K, cu_in, st);
        default: return strip_step_cs<S, kCostF32>(P, A, B, aniso, K, cu_in, st);
    }
}

cudaError_t potts_strip_step(int storage, const PottsProblem& P, const PottsStateV& a,
                             const PottsStateV& b, bool aniso, const AdmmCoef& K, float cu_in,
                             cudaStream_t st) {
    switch (storage) {
        case CMF_F32: return strip_step_s<float>(P, a, b, aniso, K, cu_in, st);
        case CMF_F16: return strip_step_s<__half>(P, a, b, aniso, K, cu_in, st);
        default: return strip_step_s<__nv_bfloat16>(P, a, b, aniso, K, cu_in, st);
    }
}

cudaError_t potts_strip_finalize(int storage, const PottsProblem& P, const PottsStateV& s,
                                 float cu, cudaStream_t st) {
    (void)storage;  // p_s is float32 for every flow storage
    const Grid& G = P.g;
    const dim3 grid((G.W + 127) / 128, G.H);
    k_potts_strip_finalize<<<grid, 128, 0, st>>>(G, P.L, s.u, s.ps, cu);
    return cudaGetLastError();
}

// ---- certificates by warp strips (Eq. relaxed-potts, Eq. potts-mf) ---------
//
// Same strips as the iteration, bands of at most kEvalRmax rows.  Phase 1
// walks the band's rows (and the row below) once over all labels: the simplex
// threshold theta of every pixel (Michelot's active-set iteration, as in the
// tile kernel) and, for rPDRQ, sum_i u_i; both go to shared memory.  Phase 2
// walks the labels, streaming each label down the band: the primal energy at
// max(u_i - theta, 0), the conservation residual of the flows y and the
// running minimum over labels of C_i + div P_alpha(y_i) (shared memory).  Sums
// are double-float per lane and per warp, FP64 per block into
// partials[blockIdx.x]; the grid has eval_blocks(H, W) blocks, the tile
// kernel's partial count.
namespace {
constexpr int kEvalRmax = 15;  // 4 warps x (16 + 15 + 15) rows x 256 B = 46 KB static
}  // namespace

template <typename S, bool ANISO, bool DR>
__global__ void __launch_bounds__(kStripWarps * 32)
    k_potts_eval_strip(PottsProblem P, PottsState<S> s, float tau, int R, int nstrips,
                       int nitems, double* partials, EvalTail T) {
    using PS = Pair<S>;
    using PF = Pair<float>;
    __shared__ float2 th_s[kStripWarps][kEvalRmax + 1][32];
    __shared__ float2 us_s[kStripWarps][kEvalRmax][32];
    __shared__ float2 dm_s[kStripWarps][kEvalRmax][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const Grid G = P.g;
    const int L = P.L;
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
        auto ld_f = [&](const float* base, int r) {
            return ok_row(r) ? PF::ld(base + r * G.pitch + c) : PF::zero();
        };
        auto ld_al = [&](int r) {
            if (!P.alpha.plane) return make_float2(P.alpha.value, P.alpha.value);
            return ld_f(P.alpha.plane, r);
        };
        auto row_w = [&](int r) { return r < G.H - 1 ? 1.f : 0.f; };

        // phase 1: theta of rows r0 .. r1 (the row below the band enters the
        // y differences of row r1-1), sum_i u_i of the band's rows
        for (int t = r0; t <= r1; ++t) {
            float2 th = make_float2(0.f, 0.f), us = make_float2(0.f, 0.f);
            if (ok_row(t)) {
                const float* ub = s.u + t * G.pitch + c;
                float sx = 0.f, sy = 0.f;
                for (int l = 0; l < L; ++l) {
                    const float2 v = PF::ld(ub + (size_t)l * G.plane);
                    sx += v.x;
                    sy += v.y;
                }
                us = make_float2(sx, sy);
                // Michelot: theta = (sum_active - 1) / n_active, active = the
                // entries above theta (the thresholds never decrease, so each
                // pass sums and counts that set afresh); stop when the counts
                // no longer change
                int nx = L, ny = L;
                float tx = (sx - 1.f) / (float)nx, ty = (sy - 1.f) / (float)ny;
                for (int it = 0; it < L; ++it) {
                    float ax = 0.f, ay = 0.f;
                    int mx = 0, my = 0;
                    for (int l = 0; l < L; ++l) {
                        const float2 v = PF::ld(ub + (size_t)l * G.plane);
                        if (v.x > tx) {
                            ax += v.x;
                            ++mx;
                        }
                        if (v.y > ty) {
                            ay += v.y;
                            ++my;
                        }
                    }
                    const bool cx = mx != nx && mx > 0, cy = my != ny && my > 0;
                    if (!cx && !cy) break;
                    if (cx) {
                        nx = mx;
                        tx = (ax - 1.f) / (float)nx;
                    }
                    if (cy) {
                        ny = my;
                        ty = (ay - 1.f) / (float)ny;
                    }
                }
                th = make_float2(tx, ty);
            }
            th_s[wib][t - r0][lane] = th;
            if (t < r1) us_s[wib][t - r0][lane] = us;
        }
        __syncwarp();

        // phase 2: per label, stream down the band; row t+1's inputs (and u of
        // row t+2) are in flight while row t is summed, stored pairs kept in
        // their storage type until used
        using SP = typename PS::T;
        struct RowIn {
            SP qx, qy, p;
            float2 c, ps, al;
            __half2 ch;  // float16 cost planes
        };
        for (int l = 0; l < L; ++l) {
            const size_t lo = (size_t)l * G.plane;
            const float* ul = s.u + lo;
            const S* qxl = s.qx + lo;
            const S* qyl = s.qy + lo;
            const float* Cb = P.lev ? P.C : P.C + lo;
            const float lev_l = P.lev ? __ldg(P.lev + l) : 0.f;
            auto ld_raw = [&](const S* base, int r) {
                return ok_row(r) ? PS::ld(base + r * G.pitch + c) : PS::zero();
            };
            auto row_in = [&](int r) {
                RowIn x;
                x.qx = ld_raw(qxl, r);
                x.qy = ld_raw(qyl, r);
                x.p = ld_raw(s.p + lo, r);
                x.ps = ld_f(s.ps, r);
                x.al = ld_al(r);
                if (P.C16) {
                    x.ch = ok_row(r) ? Pair<__half>::ld(P.C16 + lo + r * G.pitch + c)
                                     : Pair<__half>::zero();
                    x.c = PF::zero();
                } else {
                    x.c = ld_f(Cb, r);
                    x.ch = Pair<__half>::zero();
                }
                return x;
            };
            // flows y of row r (zero outside the grid); every lane shuffles
            auto flows = [&](const RowIn& x, int r, float2 u_r, float2 u_d, float2& f_x,
                             float2& f_y) {
                f_x = PS::f2(x.qx);
                f_y = PS::f2(x.qy);
                const float u_right = __shfl_down_sync(full, u_r.x, 1);
                if (DR) {
                    const float wy = row_w(r);
                    f_x.x -= tau * (u_r.y - u_r.x);
                    f_x.y -= tau * mxo * (u_right - u_r.y);
                    f_y.x -= tau * wy * (u_d.x - u_r.x);
                    f_y.y -= tau * wy * (u_d.y - u_r.y);
                }
                if (!ok_row(r)) f_x = f_y = make_float2(0.f, 0.f);
            };
            float2 u_t = ld_f(ul, r0 - 1), u_n = ld_f(ul, r0);
            float2 fx, fy;
            const RowIn x0 = row_in(r0 - 1);
            flows(x0, r0 - 1, u_t, u_n, fx, fy);
            float2 fy_up = fy, py_up;
            project_sel<ANISO>(fx.x, fy.x, x0.al.x);
            project_sel<ANISO>(fx.y, fy.y, x0.al.y);
            py_up = fy;
            u_t = u_n;
            RowIn nx = row_in(r0);
            float2 u_nn = ld_f(ul, r0 + 1);
            float2 th_t = th_s[wib][0][lane];
            for (int t = r0; t < r1; ++t) {
                const RowIn x = nx;
                u_n = u_nn;  // row t+1
                if (t + 1 < r1) nx = row_in(t + 1);
                if (t + 2 <= r1) u_nn = ld_f(ul, t + 2);
                const float2 th_n = th_s[wib][t + 1 - r0][lane];
                float2 Cl = P.C16 ? Pair<__half>::f2(x.ch) : x.c;
                if (P.lev && ok_row(t)) {
                    Cl.x = (Cl.x - lev_l) * (Cl.x - lev_l);
                    Cl.y = (Cl.y - lev_l) * (Cl.y - lev_l);
                }
                float2 fp = PS::f2(x.p), fs = x.ps;
                const float2 al = x.al;
                flows(x, t, u_t, u_n, fx, fy);
                const float wy = row_w(t);
                // primal energy at ub_i = max(u_i - theta, 0)
                const float ub_e = fmaxf(u_t.x - th_t.x, 0.f);
                const float ub_o = fmaxf(u_t.y - th_t.y, 0.f);
                const float ub_r = __shfl_down_sync(full, ub_e, 1);
                const float gx_e = ub_o - ub_e, gx_o = mxo * (ub_r - ub_o);
                const float gy_e = wy * (fmaxf(u_n.x - th_n.x, 0.f) - ub_e);
                const float gy_o = wy * (fmaxf(u_n.y - th_n.y, 0.f) - ub_o);
                const float tv_e =
                    ANISO ? fabsf(gx_e) + fabsf(gy_e) : sqrtf(gx_e * gx_e + gy_e * gy_e);
                const float tv_o =
                    ANISO ? fabsf(gx_o) + fabsf(gy_o) : sqrtf(gx_o * gx_o + gy_o * gy_o);
                const float e = (ub_e * Cl.x + al.x * tv_e) + (ub_o * Cl.y + al.y * tv_o);
                // conservation residual of y
                if (DR) {
                    const float2 us = us_s[wib][t - r0][lane];
                    fp.x += tau * u_t.x;
                    fp.y += tau * u_t.y;
                    fs.x -= tau * us.x;
                    fs.y -= tau * us.y;
                }
                const float fxl = __shfl_up_sync(full, fx.y, 1);
                const float r_e = fx.x - fxl + wy * fy.x - fy_up.x - fs.x + fp.x;
                const float r_o = mxo * fx.y - fx.x + wy * fy.y - fy_up.y - fs.y + fp.y;
                // C_i + div P_alpha(y_i), running minimum over the labels
                float px = fx.x, py = fy.x, qx_ = fx.y, qy_ = fy.y;
                project_sel<ANISO>(px, py, al.x);
                project_sel<ANISO>(qx_, qy_, al.y);
                const float pxl = __shfl_up_sync(full, qx_, 1);
                const float dp_e = px - pxl + wy * py - py_up.x;
                const float dp_o = mxo * qx_ - px + wy * qy_ - py_up.y;
                float2& dm = dm_s[wib][t - r0][lane];
                const float2 cand = make_float2(Cl.x + dp_e, Cl.y + dp_o);
                dm = l == 0 ? cand : make_float2(fminf(dm.x, cand.x), fminf(dm.y, cand.y));
                if (own) {
                    df_add(accE, e);
                    df_add(accR, r_e * r_e + r_o * r_o);
                }
                fy_up = fy;
                py_up = make_float2(py, qy_);
                u_t = u_n;
                th_t = th_n;
            }
        }
        if (own)
            for (int t = r0; t < r1; ++t) {
                const float2 dm = dm_s[wib][t - r0][lane];
                df_add(accD, dm.x + dm.y);
            }
        __syncwarp();
    }
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
static cudaError_t launch_potts_eval_strip(const PottsProblem& P, const PottsState<S>& s,
                                           float tau, double* partials, cudaStream_t st,
                                           const EvalTail& T) {
    const Grid& G = P.g;
    // the grid is eval_blocks(H, W) blocks (the partial count every
    // certificate path shares); bands sized for the warps actually resident
    const int blocks = eval_blocks(G.H, G.W);
    static std::atomic<long long> memo[kMaxDevices];  // warps resident per device
    const long long resident = strip::resident_warps(memo, k_potts_eval_strip<S, ANISO, DR>);
    const long long slots = resident > 0 ? resident : (long long)blocks * kStripWarps;
    const int nstrips = (G.W + kStripOut - 1) / kStripOut;
    const int R = strip::choose_rows(G.H, nstrips, slots, 4, kEvalRmax, 2);
    const int nitems = nstrips * ((G.H + R - 1) / R);
    k_potts_eval_strip<S, ANISO, DR>
        <<<blocks, kStripWarps * 32, 0, st>>>(P, s, tau, R, nstrips, nitems, partials, T);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t potts_eval_strip_s(const PottsProblem& P, const PottsStateV& sv, bool aniso,
                                      bool dr, float tau, double* partials, cudaStream_t st,
                                      const EvalTail& T) {
    const PottsState<S> s = sv.as<S>();
    if (dr)
        return aniso ? launch_potts_eval_strip<S, true, true>(P, s, tau, partials, st, T)
                     : launch_potts_eval_strip<S, false, true>(P, s, tau, partials, st, T);
    return aniso ? launch_potts_eval_strip<S, true, false>(P, s, tau, partials, st, T)
                 : launch_potts_eval_strip<S, false, false>(P, s, tau, partials, st, T);
}

cudaError_t potts_eval_strip(int storage, const PottsProblem& P, const PottsStateV& s,
                             bool aniso, bool dr, float tau, double* partials,
                             cudaStream_t st, const EvalTail& T) {
    switch (storage) {
        case CMF_F32: return potts_eval_strip_s<float>(P, s, aniso, dr, tau, partials, st, T);
        case CMF_F16: return potts_eval_strip_s<__half>(P, s, aniso, dr, tau, partials, st, T);
        default: return potts_eval_strip_s<__nv_bfloat16>(P, s, aniso, dr, tau, partials, st, T);
    }
}

}  // namespace cmf
