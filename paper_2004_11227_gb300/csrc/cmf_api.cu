// C-ABI layer of libcmf: argument validation, workspace layout, the
// iteration / certificate / solve drivers.  See include/cmf.h for the
// contract of every entry point.
#include <math.h>
#include <string.h>

#include <initializer_list>
#include <mutex>
#include <vector>

#include "cmf_kernels.cuh"
#include "cmf_tma.cuh"

using namespace cmf;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Workspace regions (offsets from the workspace base).
struct WsLayout {
    size_t phase;     // two state sets in phase_storage (two-phase Potts solves)
    size_t phase_set; // bytes of one of them
    size_t state;     // second state buffer set (ping-pong of the fused form)
    size_t state2;    // third set (binary fused form: routes two-iteration launches)
    size_t tmp;       // float planes used by the plain form
    size_t usum;      // two float planes of sum_i u_i (Potts rPDRQ by warp strips)
    size_t partials;  // 3 doubles per certificate block
    size_t scalars;   // 4 doubles
    size_t ctl;       // solve-loop control block (graph path)
    size_t hist;      // device history rows (graph path)
    size_t total;
};

size_t hist_rows_for(const cmf_params& p);

WsLayout ws_layout(int H, int W, int L, int pitch, const cmf_params& p, bool potts) {
    const size_t plane = (size_t)H * (size_t)pitch;
    const size_t es = dtype_size(p.storage);
    // one state set: u planes (float32), flow planes in the storage type, and
    // for Potts the float32 p_s plane; the Potts per-label planes are packed
    // [L][H][pitch]
    const size_t set = potts ? align_up(plane * 4 * L) + 3 * align_up(plane * es * L) +
                                   align_up(plane * 4)
                             : align_up(plane * 4) + 4 * align_up(plane * es);
    WsLayout w;
    size_t off = 0;
    w.phase = off;
    w.phase_set = 0;
    if (potts && p.phase_storage != 0) {
        const size_t ep = dtype_size(p.phase_storage);
        w.phase_set = align_up(plane * 4 * L) + 3 * align_up(plane * ep * L) + align_up(plane * 4);
        off += 2 * w.phase_set;
    }
    w.state = off;
    off += set;
    w.state2 = off;
    if (!potts && p.impl == CMF_FUSED) off += set;
    w.tmp = off;
    // plain forms: g and div q^{k+1} (per label for Potts); the fused kernels
    // keep everything on chip
    off += align_up(plane * 4 * (size_t)(p.impl == CMF_PLAIN ? (potts ? 2 * L : 2) : 0));
    w.usum = off;
    // fused Potts rPDRQ: each launch writes sum_i u_i of its output for the
    // next launch (ping-pong)
    if (potts && p.algo == CMF_RPDRQ && p.impl == CMF_FUSED) off += 2 * align_up(plane * 4);
    w.partials = off;
    {
        // one triple per certificate block: the certificate kernels' grid, or
        // the two-iteration launch that certifies its result
        const size_t nb = (size_t)eval_blocks(H, W);
        const size_t nc = (!potts && p.impl == CMF_FUSED) ? (size_t)binary_cert_max_blocks() : 0;
        off += align_up(sizeof(double) * 3 * (nb > nc ? nb : nc));
    }
    w.scalars = off;
    off += align_up(sizeof(double) * 4);
    w.ctl = off;
    off += align_up(64);
    w.hist = off;
    off += align_up(sizeof(double) * 5 * hist_rows_for(p));
    w.total = off;
    return w;
}

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

cmf_status check_params(const cmf_params* p, int L) {
    if (!p) return CMF_EINVAL;
    if (p->algo < CMF_PADMM || p->algo > CMF_CP) return CMF_EINVAL;
    if (p->storage < CMF_F32 || p->storage > CMF_BF16) return CMF_EINVAL;
    if (p->impl != CMF_FUSED && p->impl != CMF_PLAIN) return CMF_EINVAL;
    if (p->sweeps < 1 || (p->impl == CMF_FUSED && p->sweeps > 4) || p->sweeps > 64)
        return CMF_EINVAL;
    if (!(p->c > 0) || !(p->a > 0) || !(p->a1 > 0) || !(p->a2 >= 0)) return CMF_EINVAL;
    if (!(p->rho > 0) || !(p->rho < 2)) return CMF_EINVAL;
    if (!(p->r > 0) || !(p->sigma > 0) || !(p->tau > 0)) return CMF_EINVAL;
    if (p->max_iter < 0 || p->check_every < 1 || !(p->tol_gap >= 0)) return CMF_EINVAL;
    if (p->variant != 0 && p->variant != 1 && p->variant != 2 && p->variant != 4 &&
        p->variant != 8 && p->variant != 16 && p->variant != 32)
        return CMF_EINVAL;
    if (p->costs < 0 || p->costs > 2) return CMF_EINVAL;
    if (p->tune_step != 0 && p->tune_step != 1) return CMF_EINVAL;
    // two-phase Potts solves: a 16-bit first phase, the caller's buffers float32
    if (p->phase_storage < 0 || p->phase_storage > CMF_BF16) return CMF_EINVAL;
    if (p->phase_storage != 0 &&
        (p->storage != CMF_F32 || !(p->phase_gap > p->tol_gap) || p->rho_schedule_len != 0 ||
         p->warm_start != 0))
        return CMF_EINVAL;
    // relaxation schedule {rho_k}: non-decreasing in (0, 2) (Thm 1, Thm 2),
    // continued by rho, for the two relaxed algorithms only
    if (p->rho_schedule_len < 0) return CMF_EINVAL;
    if (p->rho_schedule_len > 0) {
        if (!p->rho_schedule) return CMF_EINVAL;
        if (p->algo != CMF_RPADMM_EB && p->algo != CMF_RPDRQ) return CMF_EINVAL;
        double prev = 0.0;
        for (int k = 0; k < p->rho_schedule_len; ++k) {
            const double r = p->rho_schedule[k];
            if (!(r > 0) || !(r < 2) || !(r >= prev)) return CMF_EINVAL;
            prev = r;
        }
        if (!(prev <= p->rho)) return CMF_EINVAL;
    }
    (void)L;
    return CMF_OK;
}

cmf_status check_grid(int H, int W, int pitch) {
    if (H < 1 || W < 1 || pitch < W) return CMF_EINVAL;
    if ((double)H * (double)pitch > 4.0e12) return CMF_EINVAL;
    return CMF_OK;
}

Alpha make_alpha(const float* d_alpha, float alpha0) { return Alpha{d_alpha, alpha0}; }

Grid make_grid(int H, int W, int pitch) {
    return Grid{H, W, pitch, (size_t)H * (size_t)pitch};
}

// The Potts problem as the kernels see it.  costs == 1: d_C holds the image
// plane followed by the L levels; costs == 2: d_C holds L float16 planes.
PottsProblem potts_problem(const float* C, int L, const float* alpha, float alpha0, int H,
                           int W, int pitch, int costs) {
    PottsProblem P{C, L, make_alpha(alpha, alpha0), make_grid(H, W, pitch), nullptr, nullptr};
    if (costs == 1) P.lev = C + (size_t)H * (size_t)pitch;
    if (costs == 2) P.C16 = reinterpret_cast<const __half*>(C);
    return P;
}

StepConfig make_step(const cmf_params& p, int L, bool potts) {
    StepConfig s;
    s.dr = p.algo == CMF_RPDRQ;
    s.aniso = p.aniso != 0;
    s.plain = p.impl == CMF_PLAIN;
    s.ac = make_admm_coef(p, L);
    s.dc = make_dr_coef(p, L, potts);
    return s;
}

// Coefficients of iteration k (counted from the start of the call): the
// scheduled rho_k where the schedule covers k, else the call's own.
StepConfig step_at(const StepConfig& base, const cmf_params& p, int L, bool potts, int k) {
    if (k >= p.rho_schedule_len) return base;
    cmf_params q = p;
    q.rho = p.rho_schedule[k];
    return make_step(q, L, potts);
}

// ---- binary ---------------------------------------------------------------

BinStateV ws_binary_state(char* ws, size_t off, const Grid& G, int storage) {
    const size_t plane = G.plane;
    const size_t es = dtype_size(storage);
    char* base = ws + off;
    BinStateV s;
    s.u = (float*)base;
    base += align_up(plane * 4);
    void** f[4] = {&s.qx, &s.qy, &s.ps, &s.pt};
    for (int i = 0; i < 4; ++i) {
        *f[i] = base;
        base += align_up(plane * es);
    }
    return s;
}

cudaError_t copy_plane(void* dst, const void* src, const Grid& G, size_t es, cudaStream_t st) {
    if (dst == src) return cudaSuccess;
    return cudaMemcpy2DAsync(dst, G.pitch * es, src, G.pitch * es, G.W * es, G.H,
                             cudaMemcpyDeviceToDevice, st);
}

cudaError_t copy_binary(const BinStateV& dst, const BinStateV& src, const Grid& G, int storage,
                        cudaStream_t st) {
    const size_t es = dtype_size(storage);
    cudaError_t e;
    if ((e = copy_plane(dst.u, src.u, G, 4, st)) != cudaSuccess) return e;
    if ((e = copy_plane(dst.qx, src.qx, G, es, st)) != cudaSuccess) return e;
    if ((e = copy_plane(dst.qy, src.qy, G, es, st)) != cudaSuccess) return e;
    if ((e = copy_plane(dst.ps, src.ps, G, es, st)) != cudaSuccess) return e;
    return copy_plane(dst.pt, src.pt, G, es, st);
}

struct BinaryCall {
    BinProblem P;
    BinStateV user, ws, ws2;  // buffer sets 0, 1, 2 (set 2: fused form only)
    WsLayout w;
    char* wsbase;
    StepConfig cfg;
    cmf_params prm;         // the call's parameters (rho schedule)
    int storage;
    bool tma;               // fused ADMM through the persistent TMA kernel
    bool strip;             // fused ADMM by warp strips
    bool pairs;             // warp strips, two ADMM iterations per launch
    BinTmaMaps maps[2];     // tensor maps of the user / workspace state sets
    int* err;               // sticky device error word
};

cmf_status binary_prepare(const float* Cs, const float* Ct, const float* alpha, float alpha0,
                          int H, int W, int pitch, const cmf_params* p, float* u, void* qx,
                          void* qy, void* ps, void* pt, void* ws, size_t ws_bytes,
                          BinaryCall& call) {
    cmf_status s;
    if ((s = check_params(p, 2)) != CMF_OK) return s;
    if (p->costs != 0) return CMF_EINVAL;  // binary costs are planes
    if (p->phase_storage != 0) return CMF_EINVAL;  // two-phase solves: Potts only
    if ((s = check_grid(H, W, pitch)) != CMF_OK) return s;
    if (!Cs || !Ct || !u || !qx || !qy || !ps || !pt || !ws) return CMF_EINVAL;
    if (!alpha && !(alpha0 >= 0.0f && isfinite(alpha0))) return CMF_EINVAL;
    const size_t es = dtype_size(p->storage);
    if (!aligned(u, 4) || !aligned(Cs, 4) || !aligned(Ct, 4) || (alpha && !aligned(alpha, 4)))
        return CMF_EINVAL;
    if (!aligned(qx, es) || !aligned(qy, es) || !aligned(ps, es) || !aligned(pt, es))
        return CMF_EINVAL;
    if (!aligned(ws, kAlign)) return CMF_EINVAL;
    call.w = ws_layout(H, W, 2, pitch, *p, false);
    if (ws_bytes < call.w.total) return CMF_ENOMEM;
    call.P = BinProblem{Cs, Ct, make_alpha(alpha, alpha0), make_grid(H, W, pitch)};
    call.user = BinStateV{u, qx, qy, ps, pt};
    call.wsbase = (char*)ws;
    call.ws = ws_binary_state(call.wsbase, call.w.state, call.P.g, p->storage);
    call.ws2 = ws_binary_state(call.wsbase, call.w.state2, call.P.g, p->storage);
    call.cfg = make_step(*p, 2, false);
    call.prm = *p;
    call.storage = p->storage;
    call.err = &((SolveCtl*)(call.wsbase + call.w.ctl))->err;
    call.tma = false;
    call.strip = false;
    call.pairs = false;
    // automatic choice: warp strips where the layout allows them, two ADMM
    // iterations per launch (1.5x faster per iteration than one at 1024^2,
    // 1.9x at 4096^2, which beats the persistent TMA kernel: measured);
    // rPDRQ: the pipelined red-black sweeps
    if (!call.cfg.plain && (p->variant == 2 || p->variant == 4 || p->variant == 0)) {
        const bool ok =
            binary_strip_eligible(call.P.g, p->storage, Cs, Ct, alpha, call.user, call.ws);
        if (!ok && p->variant != 0)
            return CMF_EINVAL;  // warp strips requested but the layout does not allow them
        if (ok) {
            call.strip = true;
            call.pairs = p->variant != 2 && !call.cfg.dr;
            return CMF_OK;
        }
    }
    const int ty = p->variant >= 8 ? p->variant : 16;
    // automatic choice: the persistent TMA kernel wins on grids that fit the
    // L2 cache, the shared-memory tile kernel on larger ones (measured)
    const bool auto_tma = p->variant == 0 && (size_t)H * (size_t)W <= ((size_t)1 << 21);
    if (!call.cfg.dr && !call.cfg.plain && (p->variant >= 8 || auto_tma) &&
        binary_tma_eligible(call.P.g, p->storage, call.user) &&
        binary_tma_eligible(call.P.g, p->storage, call.ws)) {
        call.tma = binary_tma_maps(call.P.g, p->storage, call.user, ty, call.maps[0]) ==
                       cudaSuccess &&
                   binary_tma_maps(call.P.g, p->storage, call.ws, ty, call.maps[1]) ==
                       cudaSuccess;
    }
    if (!call.tma && !call.cfg.dr && !call.cfg.plain && p->variant >= 8)
        return CMF_EINVAL;  // TMA tiles requested but the layout does not allow them
    return CMF_OK;
}

const BinStateV& bset(const BinaryCall& c, int i) {
    return i == 0 ? c.user : (i == 1 ? c.ws : c.ws2);
}

// Run n iterations starting from `cur` (0 = user buffers, 1 = workspace,
// 2 = the workspace's third set, used by the two-iteration launches);
// returns the index of the buffer set holding the result.  k0 is the index of
// the first of them within the call (for the rho schedule).  cert != nullptr:
// also certify the result with that tail (in the last two-iteration launch
// when there is one, else with the certificate kernel).  dry: launch
// nothing, only follow the buffer sets.
cudaError_t binary_run(const BinaryCall& c, int n, int& cur, cudaStream_t st, int k0 = 0,
                       const EvalTail* cert = nullptr, bool dry = false) {
    float* tmp = (float*)(c.wsbase + c.w.tmp);
    double* partials = (double*)(c.wsbase + c.w.partials);
    bool certified = false;
    // Two-iteration launches after the scheduled iterations (one single
    // launch for an odd remainder).  With three buffer sets a run of at least
    // two launches ends in the set it started from: start -> x -> y -> x ...
    // -> start, x and y the other two sets; a lone launch goes to the
    // caller's set, or from it to the workspace.
    int i = 0;
    if (c.pairs) {
        const int sched = c.prm.rho_schedule_len > k0 ? c.prm.rho_schedule_len - k0 : 0;
        const int first = sched < n ? sched : n;
        for (; i < first; ++i) {
            const StepConfig cfg = step_at(c.cfg, c.prm, 2, false, k0 + i);
            const int dst = cur == 0 ? 1 : 0;
            if (!dry) {
                cudaError_t e = binary_strip_step(c.storage, c.P, bset(c, cur), bset(c, dst),
                                                  cfg.aniso, cfg.ac, st);
                if (e != cudaSuccess) return e;
            }
            cur = dst;
        }
        const int npairs = (n - first) / 2, nsingle = (n - first) % 2;
        const int nl = npairs + nsingle;
        const int start = cur;
        const int x = start == 0 ? 1 : 0, y = start == 2 ? 1 : 2;
        for (int j = 0; j < nl; ++j) {
            const int dst = nl == 1 ? (start == 0 ? 1 : 0)
                                    : (j == nl - 1 ? start : (j % 2 == 0 ? x : y));
            // the last pair launch carries the certificates when no single follows it
            const bool cj = cert && j == npairs - 1 && nsingle == 0;
            if (!dry) {
                const BinStateV& a = bset(c, cur);
                const BinStateV& b = bset(c, dst);
                cudaError_t e =
                    j < npairs ? binary_strip2_step(c.storage, c.P, a, b, c.cfg.aniso, c.cfg.ac,
                                                    st, cj ? cert : nullptr, partials)
                               : binary_strip_step(c.storage, c.P, a, b, c.cfg.aniso, c.cfg.ac,
                                                   st);
                if (e != cudaSuccess) return e;
            }
            certified = certified || cj;
            cur = dst;
        }
        i = n;
    }
    for (; i < n; ++i) {
        const StepConfig cfg = step_at(c.cfg, c.prm, 2, false, k0 + i);
        if (cfg.plain) {
            if (!dry) {
                cudaError_t e = binary_step(c.storage, c.P, c.user, c.user, cfg, tmp, st);
                if (e != cudaSuccess) return e;
            }
            cur = 0;
        } else if (c.strip) {
            const BinStateV& a = cur == 0 ? c.user : c.ws;
            const BinStateV& b = cur == 0 ? c.ws : c.user;
            if (!dry) {
                cudaError_t e =
                    cfg.dr ? binary_dr_strip_step(c.storage, c.P, a, b, cfg.aniso, cfg.dc, st)
                           : binary_strip_step(c.storage, c.P, a, b, cfg.aniso, cfg.ac, st);
                if (e != cudaSuccess) return e;
            }
            cur ^= 1;
        } else if (c.tma) {
            const BinStateV& b = cur == 0 ? c.ws : c.user;
            if (!dry) {
                cudaError_t e = binary_admm_tma_step(c.storage, c.P, b, cfg.aniso, cfg.ac,
                                                     c.maps[cur], c.err, st);
                if (e != cudaSuccess) return e;
            }
            cur ^= 1;
        } else {
            const BinStateV& a = cur == 0 ? c.user : c.ws;
            const BinStateV& b = cur == 0 ? c.ws : c.user;
            if (!dry) {
                cudaError_t e = binary_step(c.storage, c.P, a, b, cfg, tmp, st);
                if (e != cudaSuccess) return e;
            }
            cur ^= 1;
        }
    }
    if (cert && !certified && !dry)
        return binary_eval(c.storage, c.P, bset(c, cur), c.cfg.aniso, c.cfg.dr, c.cfg.dc.tau,
                           partials, st, *cert);
    return cudaSuccess;
}

// The certificate launch has reduced its partials into the scalars (its last
// block); read them and the error word.
cmf_status finish_eval(char* wsbase, const WsLayout& w, double* h_out, cudaStream_t st) {
    double* scal = (double*)(wsbase + w.scalars);
    double h[3];
    CMF_CUDA_TRY(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, st));
    int* err = &((SolveCtl*)(wsbase + w.ctl))->err;
    int herr = 0;
    CMF_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CMF_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr == kErrWaitTimeout) {
        CMF_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        return CMF_ETIMEOUT;
    }
    const double E = h[0], D = h[1];
    h_out[0] = E;
    h_out[1] = D;
    h_out[2] = (E - D) / (fabs(E) > 1e-30 ? fabs(E) : 1e-30);
    h_out[3] = sqrt(h[2] > 0 ? h[2] : 0.0);
    return CMF_OK;
}

// The certificate launch with its own reduction (no stop decision).
EvalTail reduce_tail(char* wsbase, const WsLayout& w) {
    EvalTail T;
    T.ctl = (SolveCtl*)(wsbase + w.ctl);
    T.scal = (double*)(wsbase + w.scalars);
    return T;
}

cmf_status binary_eval_state(const BinaryCall& c, const BinStateV& s, double* h_out,
                             cudaStream_t st) {
    const EvalTail T = reduce_tail(c.wsbase, c.w);
    CMF_CUDA_TRY(cudaMemsetAsync(&T.ctl->arrive, 0, sizeof(unsigned), st));
    CMF_CUDA_TRY(binary_eval(c.storage, c.P, s, c.cfg.aniso, c.cfg.dr, c.cfg.dc.tau,
                             (double*)(c.wsbase + c.w.partials), st, T));
    return finish_eval(c.wsbase, c.w, h_out, st);
}

// ---- Potts ----------------------------------------------------------------

PottsStateV ws_potts_state(char* ws, size_t off, const Grid& G, int L, int storage) {
    const size_t plane = G.plane;
    const size_t es = dtype_size(storage);
    char* base = ws + off;
    PottsStateV s;
    s.u = (float*)base;
    base += align_up(plane * 4 * L);
    s.qx = base;
    base += align_up(plane * es * L);
    s.qy = base;
    base += align_up(plane * es * L);
    s.p = base;
    base += align_up(plane * es * L);
    s.ps = (float*)base;
    return s;
}

cudaError_t copy_potts(const PottsStateV& dst, const PottsStateV& src, const Grid& G, int L,
                       int storage, cudaStream_t st) {
    const size_t es = dtype_size(storage);
    cudaError_t e;
    for (int i = 0; i < L; ++i) {
        const size_t o4 = G.plane * 4 * i, oe = G.plane * es * i;
        if ((e = copy_plane((char*)dst.u + o4, (char*)src.u + o4, G, 4, st)) != cudaSuccess)
            return e;
        if ((e = copy_plane((char*)dst.qx + oe, (char*)src.qx + oe, G, es, st)) != cudaSuccess)
            return e;
        if ((e = copy_plane((char*)dst.qy + oe, (char*)src.qy + oe, G, es, st)) != cudaSuccess)
            return e;
        if ((e = copy_plane((char*)dst.p + oe, (char*)src.p + oe, G, es, st)) != cudaSuccess)
            return e;
    }
    return copy_plane(dst.ps, src.ps, G, 4, st);  // p_s: float32
}

struct PottsCall {
    PottsProblem P;
    PottsStateV user, ws;
    WsLayout w;
    char* wsbase;
    StepConfig cfg;
    cmf_params prm;              // the call's parameters (rho schedule)
    int storage;
    bool tma;                    // fused ADMM through TMA-staged tiles
    bool strip;                  // fused ADMM by warp strips
    PottsTmaMaps maps[2];        // tensor maps of the user / workspace state sets
    int* err;                    // sticky device error word
};

// `layout`: the parameters the workspace was sized for (default *p); `set`:
// the second state set (default: the workspace's own, in p->storage).
cmf_status potts_prepare(const float* C, int L, const float* alpha, float alpha0, int H, int W,
                         int pitch, const cmf_params* p, float* u, void* qx, void* qy, void* pp,
                         void* ps, void* ws, size_t ws_bytes, PottsCall& call,
                         const cmf_params* layout = nullptr, const PottsStateV* set = nullptr) {
    cmf_status s;
    if (L < 2 || L > 64) return CMF_EINVAL;
    if ((s = check_params(p, L)) != CMF_OK) return s;
    if ((s = check_grid(H, W, pitch)) != CMF_OK) return s;
    if (!C || !u || !qx || !qy || !pp || !ps || !ws) return CMF_EINVAL;
    if (!alpha && !(alpha0 >= 0.0f && isfinite(alpha0))) return CMF_EINVAL;
    const size_t es = dtype_size(p->storage);
    if (!aligned(u, 4) || !aligned(C, p->costs == 2 ? 2 : 4) || (alpha && !aligned(alpha, 4)))
        return CMF_EINVAL;
    if (!aligned(qx, es) || !aligned(qy, es) || !aligned(pp, es) || !aligned(ps, 4))
        return CMF_EINVAL;
    if (!aligned(ws, kAlign)) return CMF_EINVAL;
    call.w = ws_layout(H, W, L, pitch, layout ? *layout : *p, true);
    if (ws_bytes < call.w.total) return CMF_ENOMEM;
    call.P = potts_problem(C, L, alpha, alpha0, H, W, pitch, p->costs);
    call.user = PottsStateV{u, qx, qy, pp, (float*)ps};
    call.wsbase = (char*)ws;
    call.ws = set ? *set : ws_potts_state(call.wsbase, call.w.state, call.P.g, L, p->storage);
    call.cfg = make_step(*p, L, true);
    call.prm = *p;
    call.storage = p->storage;
    call.err = &((SolveCtl*)(call.wsbase + call.w.ctl))->err;
    call.tma = false;
    call.strip = false;
    // automatic choice: warp strips where the layout allows them (fastest on
    // every measured Potts case), else TMA tiles, else shared-memory tiles
    if (!call.cfg.plain && (p->variant == 2 || p->variant == 4 || p->variant == 0)) {
        const bool ok = potts_strip_eligible(call.P.g, p->storage, C, alpha, call.user, call.ws);
        if (!ok && p->variant != 0)
            return CMF_EINVAL;  // warp strips requested but the layout does not allow them
        if (ok) {
            call.strip = true;
            return CMF_OK;
        }
    }
    const bool want_tma = !call.cfg.dr && !call.cfg.plain && p->variant != 1;
    const int ty = p->variant >= 8 ? p->variant
                                   : (want_tma ? potts_tma_auto_ty(p->storage, p->aniso, L) : 16);
    if (want_tma && potts_tma_fits(p->storage, L, ty) &&
        potts_tma_eligible(call.P.g, p->storage, call.user) &&
        potts_tma_eligible(call.P.g, p->storage, call.ws)) {
        call.tma = potts_tma_maps(call.P.g, L, p->storage, call.user, ty, call.maps[0]) ==
                       cudaSuccess &&
                   potts_tma_maps(call.P.g, L, p->storage, call.ws, ty, call.maps[1]) ==
                       cudaSuccess;
    }
    if (!call.tma && !call.cfg.dr && !call.cfg.plain && p->variant >= 8)
        return CMF_EINVAL;  // TMA tiles requested but the layout does not allow them
    return CMF_OK;
}

// As binary_run: n iterations from buffer set `cur` (0 or 1); cert: certify
// the result with that tail; dry: only follow the buffer sets.
cudaError_t potts_run(const PottsCall& c, int n, int& cur, cudaStream_t st, int k0 = 0,
                      const EvalTail* cert = nullptr, bool dry = false) {
    if (dry) {
        if (n > 0) cur = c.cfg.plain ? 0 : (n % 2 ? cur ^ 1 : cur);
        return cudaSuccess;
    }
    float* tmp = (float*)(c.wsbase + c.w.tmp);
    for (int i = 0; i < n; ++i) {
        const StepConfig cfg = step_at(c.cfg, c.prm, c.P.L, true, k0 + i);
        if (cfg.plain) {
            cudaError_t e = potts_step(c.storage, c.P, c.user, c.user, cfg, tmp, st);
            if (e != cudaSuccess) return e;
            cur = 0;
        } else if (c.strip && cfg.dr) {
            const PottsStateV& a = cur == 0 ? c.user : c.ws;
            const PottsStateV& b = cur == 0 ? c.ws : c.user;
            // sum_i u_i planes: the call's first launch sums u itself, later
            // ones read what the previous launch wrote
            float* U = (float*)(c.wsbase + c.w.usum);
            const size_t up = align_up((size_t)c.P.g.H * (size_t)c.P.g.pitch * 4) / 4;
            cudaError_t e = potts_dr_strip_step(c.storage, c.P, a, b, cfg.aniso, cfg.dc,
                                                i == 0 ? nullptr : U + cur * up,
                                                U + (cur ^ 1) * up, st);
            if (e != cudaSuccess) return e;
            cur ^= 1;
        } else if (c.strip) {
            const PottsStateV& a = cur == 0 ? c.user : c.ws;
            const PottsStateV& b = cur == 0 ? c.ws : c.user;
            // the first iteration reads u itself, later ones the w form (cu
            // does not depend on rho, so a schedule keeps it fixed)
            cudaError_t e = potts_strip_step(c.storage, c.P, a, b, cfg.aniso, cfg.ac,
                                             i == 0 ? 0.0f : cfg.ac.cu, st);
            if (e != cudaSuccess) return e;
            cur ^= 1;
            if (i == n - 1 &&
                (e = potts_strip_finalize(c.storage, c.P, b, cfg.ac.cu, st)) != cudaSuccess)
                return e;
        } else if (c.tma) {
            const PottsStateV& b = cur == 0 ? c.ws : c.user;
            cudaError_t e = potts_admm_tma_step(c.storage, c.P, b, cfg.aniso, cfg.ac,
                                                c.maps[cur], c.err, st);
            if (e != cudaSuccess) return e;
            cur ^= 1;
        } else {
            const PottsStateV& a = cur == 0 ? c.user : c.ws;
            const PottsStateV& b = cur == 0 ? c.ws : c.user;
            cudaError_t e = potts_step(c.storage, c.P, a, b, cfg, tmp, st);
            if (e != cudaSuccess) return e;
            cur ^= 1;
        }
    }
    if (cert)
        return potts_eval(c.storage, c.P, cur == 0 ? c.user : c.ws, c.cfg.aniso, c.cfg.dr,
                          c.cfg.dc.tau, (double*)(c.wsbase + c.w.partials), st, *cert);
    return cudaSuccess;
}

cmf_status potts_eval_state(const PottsCall& c, const PottsStateV& s, double* h_out,
                            cudaStream_t st) {
    const EvalTail T = reduce_tail(c.wsbase, c.w);
    CMF_CUDA_TRY(cudaMemsetAsync(&T.ctl->arrive, 0, sizeof(unsigned), st));
    CMF_CUDA_TRY(potts_eval(c.storage, c.P, s, c.cfg.aniso, c.cfg.dr, c.cfg.dc.tau,
                            (double*)(c.wsbase + c.w.partials), st, T));
    return finish_eval(c.wsbase, c.w, h_out, st);
}

// ---- device-driven solve loop (CUDA graph with a conditional WHILE node) ----

__global__ void k_solve_reset(SolveCtl* ctl, int it0) {
    ctl->it = it0;
    ctl->checks = 0;
    ctl->stop = 0;
    ctl->where = 0;
    ctl->arrive = 0;
}

// End of a two-chunk loop body: go on unless either half stopped.
__global__ void k_solve_loop_cond(const SolveCtl* ctl, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, ctl->stop == 0 ? 1u : 0u);
}

size_t hist_rows_for(const cmf_params& p) {
    const size_t r = (size_t)(p.max_iter / (p.check_every > 0 ? p.check_every : 1)) + 1;
    return r < 65536 ? r : 65536;  // later checks are decided but not recorded
}

// Whether the graph path can reproduce the host loop exactly: whole chunks
// only.  (A chunk that ends in the workspace buffers makes the loop body two
// chunks long, see solve_graph.)
bool graph_eligible(const cmf_params& p) {
    if (!p.use_graph || p.max_iter < p.check_every) return false;
    if (p.max_iter % p.check_every != 0) return false;
    return true;
}

// Everything the kernels of a solve graph are built from: the device, the
// model, sizes, every device pointer, alpha0 and the parameters (their
// coefficients, the loop constants).  Calls with equal signatures can replay
// the same instantiated graph.  Zero-filled before use (padding included) and
// filled field by field, then compared bytewise.
struct SolveSig {
    int dev, model, L, H, W, pitch;
    float alpha0;
    const void* ptr[10];
    cmf_params p;  // rho schedule and warm start cleared: the graph does not depend on them
};

SolveSig make_sig(int model, int L, int H, int W, int pitch, float alpha0,
                  std::initializer_list<const void*> ptrs, const cmf_params& p) {
    SolveSig k;
    memset(&k, 0, sizeof(k));
    cudaGetDevice(&k.dev);
    k.model = model;
    k.L = L;
    k.H = H;
    k.W = W;
    k.pitch = pitch;
    k.alpha0 = alpha0;
    int i = 0;
    for (const void* q : ptrs)
        if (i < 10) k.ptr[i++] = q;
    // field by field: the caller's padding bytes (after `costs`, at the tail)
    // stay zero, so equal parameters always compare equal
    k.p.algo = p.algo;
    k.p.storage = p.storage;
    k.p.impl = p.impl;
    k.p.aniso = p.aniso;
    k.p.sweeps = p.sweeps;
    k.p.max_iter = p.max_iter;
    k.p.check_every = p.check_every;
    k.p.use_graph = p.use_graph;
    k.p.variant = p.variant;
    k.p.c = p.c;
    k.p.a = p.a;
    k.p.a1 = p.a1;
    k.p.a2 = p.a2;
    k.p.rho = p.rho;
    k.p.r = p.r;
    k.p.sigma = p.sigma;
    k.p.tau = p.tau;
    k.p.tol_gap = p.tol_gap;
    k.p.costs = p.costs;
    k.p.phase_storage = p.phase_storage;
    k.p.phase_gap = p.phase_gap;
    k.p.tune_step = p.tune_step;
    return k;
}

// Instantiated solve graphs, least recently used out.  Graph objects stay
// alive between calls (until evicted or cmf_release_graphs); an executable
// graph that is destroyed while in flight is freed when it completes.
constexpr size_t kGraphCache = 8;
struct GraphEntry {
    SolveSig sig;
    cudaGraph_t g;
    cudaGraphExec_t ge;
    unsigned long long used;
};
std::mutex g_graph_mu;
std::vector<GraphEntry>* g_graphs = new std::vector<GraphEntry>();  // never freed: no
                                                                     // CUDA calls at exit
unsigned long long g_graph_tick = 0;

cudaGraphExec_t graph_lookup(const SolveSig& k) {
    for (GraphEntry& e : *g_graphs)
        if (memcmp(&e.sig, &k, sizeof(k)) == 0) {
            e.used = ++g_graph_tick;
            return e.ge;
        }
    return nullptr;
}

void graph_insert(const SolveSig& k, cudaGraph_t g, cudaGraphExec_t ge) {
    if (g_graphs->size() >= kGraphCache) {
        size_t lru = 0;
        for (size_t i = 1; i < g_graphs->size(); ++i)
            if ((*g_graphs)[i].used < (*g_graphs)[lru].used) lru = i;
        cudaGraphExecDestroy((*g_graphs)[lru].ge);
        cudaGraphDestroy((*g_graphs)[lru].g);
        g_graphs->erase(g_graphs->begin() + lru);
    }
    g_graphs->push_back(GraphEntry{k, g, ge, ++g_graph_tick});
}

void graph_drop(cudaGraphExec_t ge) {
    for (size_t i = 0; i < g_graphs->size(); ++i)
        if ((*g_graphs)[i].ge == ge) {
            cudaGraphExecDestroy(ge);
            cudaGraphDestroy((*g_graphs)[i].g);
            g_graphs->erase(g_graphs->begin() + i);
            return;
        }
}

// The stall test of a two-phase solve's first phase (solve_decide): off when
// iters == 0; the window is the checks that cover `iters` iterations.
struct StallRule {
    int iters = 0;
    double factor = 0.0, near = 0.0;
    int checks(int check_every) const {
        return iters > 0 ? (iters + check_every - 1) / check_every : 0;
    }
};

// `chunk(stream, from)` launches check_every iterations starting in buffer
// set `from` (0 = the caller's, 1 = the workspace's) and returns the set they
// end in through `to`; `certify(stream, set)` launches the certificate kernel
// for a set into the partials.  A chunk that ends in the caller's buffers
// makes the loop body {chunk, certificates, decide}; one that ends in the
// workspace makes it two chunks, the second under a conditional IF node that
// the first half's decision sets, and a last kernel that sets the loop's
// condition (so a solve can stop after either half; `copy_back` then brings
// the state home).  The loop continues a solve that has already run it0
// iterations and recorded nh0 history rows on the host.  The graph is built
// and instantiated on the first call with signature `sig` and replayed after.
template <typename Chunk, typename EndOf, typename Copy>
cmf_status solve_graph(const cmf_params* p, const SolveSig& sig, char* wsbase, const WsLayout& w,
                       Chunk chunk, EndOf end_of, Copy copy_back, double* h_hist,
                       int hist_cap, int* h_iters, cudaStream_t st, int it0 = 0, int nh0 = 0,
                       const StallRule& sr = StallRule()) {
    SolveCtl* ctl = (SolveCtl*)(wsbase + w.ctl);
    double* dhist = (double*)(wsbase + w.hist);
    const int rows = (int)hist_rows_for(*p);
    // the certificate launch reduces its partials and takes the stop decision
    // in its last block: one node per check
    EvalTail T = reduce_tail(wsbase, w);
    T.decide = true;
    T.hist = dhist;
    T.hist_rows = rows;
    T.K = p->check_every;
    T.max_iter = p->max_iter;
    T.tol = p->tol_gap;
    T.stall = sr.checks(p->check_every);
    T.stall_f = sr.factor;
    T.stall_near = sr.near;
    k_solve_reset<<<1, 1, 0, st>>>(ctl, it0);
    CMF_CUDA_TRY(cudaGetLastError());

    std::lock_guard<std::mutex> lock(g_graph_mu);
    cudaGraphExec_t ge = graph_lookup(sig);
    if (!ge) {
        cudaStream_t cs = nullptr, cs2 = nullptr;
        cudaGraph_t g = nullptr;
        bool ok = false;
        do {
            if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) break;
            if (cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking) != cudaSuccess) break;
            if (cudaGraphCreate(&g, 0) != cudaSuccess) break;
            cudaGraphConditionalHandle h;
            if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) !=
                cudaSuccess)
                break;
            cudaGraphNodeParams np = {};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) break;
            cudaGraph_t body = np.conditional.phGraph_out[0];
            if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed) != cudaSuccess)
                break;
            // the set a chunk from the caller's buffers ends in decides the body
            const int mid = end_of(0);
            // the IF node's handle, only when there is a second half (a handle
            // without its node fails the instantiation)
            cudaError_t e = cudaSuccess;
            cudaGraphConditionalHandle h_if = 0;
            if (mid) e = cudaGraphConditionalHandleCreate(&h_if, body, 0, cudaGraphCondAssignDefault);
            if (e == cudaSuccess) {
                EvalTail T1 = T;
                T1.h = mid ? h_if : h;
                T1.set_h = mid ? 2 : 1;
                T1.where = mid;
                int got = 0;
                e = chunk(cs, 0, got, T1);  // iterations and their certificates
                if (e == cudaSuccess && got != mid) e = cudaErrorInvalidValue;
            }
            if (e == cudaSuccess && mid) {
                // second half: an IF node on the first half's decision
                cudaStreamCaptureStatus cst;
                const cudaGraphNode_t* deps = nullptr;
                const cudaGraphEdgeData* edges = nullptr;
                size_t ndeps = 0;
                cudaGraph_t cg = nullptr;
                e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, &edges, &ndeps);
                cudaGraphNodeParams ip = {};
                ip.type = cudaGraphNodeTypeConditional;
                ip.conditional.handle = h_if;
                ip.conditional.type = cudaGraphCondTypeIf;
                ip.conditional.size = 1;
                cudaGraphNode_t ifnode;
                if (e == cudaSuccess)
                    e = cudaGraphAddNode(&ifnode, body, deps, edges, ndeps, &ip);
                if (e == cudaSuccess)
                    e = cudaStreamUpdateCaptureDependencies(cs, &ifnode, nullptr, 1,
                                                            cudaStreamSetCaptureDependencies);
                if (e == cudaSuccess)
                    e = cudaStreamBeginCaptureToGraph(cs2, ip.conditional.phGraph_out[0],
                                                      nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeRelaxed);
                if (e == cudaSuccess) {
                    int end = mid;
                    EvalTail T2 = T;  // conditions left to k_solve_loop_cond
                    cudaError_t f = chunk(cs2, mid, end, T2);
                    if (f == cudaSuccess && end != 0) f = cudaErrorInvalidValue;
                    cudaGraph_t cap2 = nullptr;
                    cudaError_t f2 = cudaStreamEndCapture(cs2, &cap2);
                    e = f != cudaSuccess ? f : f2;
                }
                if (e == cudaSuccess) {
                    k_solve_loop_cond<<<1, 1, 0, cs>>>(ctl, h);
                    e = cudaGetLastError();
                }
            }
            cudaGraph_t captured = nullptr;
            cudaError_t e4 = cudaStreamEndCapture(cs, &captured);
            if (e != cudaSuccess || e4 != cudaSuccess) break;
            if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) break;
            ok = true;
        } while (0);
        if (cs2) cudaStreamDestroy(cs2);
        if (cs) cudaStreamDestroy(cs);
        if (!ok) {
            if (ge) cudaGraphExecDestroy(ge);
            if (g) cudaGraphDestroy(g);
            return CMF_ECUDA;
        }
        graph_insert(sig, g, ge);
    }
    if (cudaGraphLaunch(ge, st) != cudaSuccess) {
        graph_drop(ge);
        return CMF_ECUDA;
    }
    SolveCtl hc;
    CMF_CUDA_TRY(cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, st));
    CMF_CUDA_TRY(cudaStreamSynchronize(st));
    const int n = hc.checks < rows ? hc.checks : rows;
    const int room = hist_cap > nh0 ? hist_cap - nh0 : 0;
    const int ncopy = n < room ? n : room;
    if (h_hist && ncopy > 0)
        CMF_CUDA_TRY(cudaMemcpy(h_hist + 5 * (size_t)nh0, dhist, sizeof(double) * 5 * (size_t)ncopy,
                                cudaMemcpyDeviceToHost));
    if (h_iters) *h_iters = hc.it;
    if (hc.where != 0) {  // stopped after the first half of a two-chunk body
        CMF_CUDA_TRY(copy_back(hc.where));
        CMF_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return hc.stop == 1 ? CMF_OK : (hc.stop == 3 ? CMF_ETIMEOUT : CMF_NOT_CONVERGED);
}

// Progress of a host-driven solve loop.
struct LoopState {
    int it = 0;    // iterations done
    int nh = 0;    // certificate checks done
    int cur = 0;   // buffer set holding the state (0 = caller's)
    bool converged = false;
};

// Host-driven chunks of check_every iterations, each with the certificates
// of its result, until convergence, max_iter, or it >= it_stop.
// `run_cert(n, cur, k0, out)` advances n iterations whose first is iteration
// k0 of the solve and writes the certificates (E, D, gap, res) to out.
template <typename RunCert>
cmf_status loop_chunks(const cmf_params* p, int it_stop, RunCert run_cert, double* h_hist,
                       int hist_cap, LoopState& ls, const StallRule& sr = StallRule()) {
    double out[4];
    const int stall = sr.checks(p->check_every);
    double gref = 0.0;  // the stall test, as solve_decide keeps it
    int nchk = 0;
    while (ls.it < p->max_iter && ls.it < it_stop) {
        const int k =
            p->check_every < p->max_iter - ls.it ? p->check_every : p->max_iter - ls.it;
        cmf_status s = run_cert(k, ls.cur, ls.it, out);
        if (s != CMF_OK) return s;
        ls.it += k;
        if (h_hist && ls.nh < hist_cap) {
            double* row = h_hist + 5 * (size_t)ls.nh;
            row[0] = ls.it;
            row[1] = out[0];
            row[2] = out[1];
            row[3] = out[2];
            row[4] = out[3];
        }
        ++ls.nh;
        bool stalled = false;
        if (stall > 0 && nchk % stall == 0) {
            stalled = nchk > 0 && out[2] < sr.near && out[2] > sr.factor * gref;
            gref = out[2];
        }
        ++nchk;
        if (out[2] <= p->tol_gap || stalled) {
            ls.converged = true;
            break;
        }
    }
    return CMF_OK;
}

template <typename Copy>
cmf_status finish_loop(const LoopState& ls, Copy copy_back, int* h_iters, cudaStream_t st) {
    if (ls.cur != 0) CMF_CUDA_TRY(copy_back(ls.cur));
    CMF_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_iters) *h_iters = ls.it;
    return ls.converged ? CMF_OK : CMF_NOT_CONVERGED;
}

// The solve driver: the iterations a rho schedule covers run host-driven
// (their coefficients change from launch to launch, a graph's are fixed), the
// rest in the device-driven graph where it applies, else host-driven.
// `chunk(stream, from, to, tail)` captures one graph chunk with its
// certificates, `end_of(from)` tells the set a chunk ends in.
// it0, nh0: iterations and history rows an earlier phase of the same solve
// has already done (the loop continues their count; max_iter is the total).
template <typename RunCert, typename Copy, typename Chunk, typename EndOf>
cmf_status solve_driver(const cmf_params* p, const SolveSig& sig, char* wsbase, const WsLayout& w,
                        RunCert run_cert, Copy copy_back, Chunk chunk, EndOf end_of,
                        double* h_hist, int hist_cap, int* h_iters, cudaStream_t st,
                        int it0 = 0, int nh0 = 0, const StallRule& sr = StallRule()) {
    LoopState ls;
    ls.it = it0;
    ls.nh = nh0;
    if (!graph_eligible(*p)) {
        cmf_status s = loop_chunks(p, p->max_iter, run_cert, h_hist, hist_cap, ls, sr);
        if (s != CMF_OK) return s;
        return finish_loop(ls, copy_back, h_iters, st);
    }
    if (p->rho_schedule_len > 0) {
        cmf_status s = loop_chunks(p, p->rho_schedule_len, run_cert, h_hist, hist_cap, ls);
        if (s != CMF_OK) return s;
        if (ls.cur != 0) CMF_CUDA_TRY(copy_back(ls.cur));  // the graph starts from set 0
        ls.cur = 0;
        if (ls.converged || ls.it >= p->max_iter) return finish_loop(ls, copy_back, h_iters, st);
    }
    return solve_graph(p, sig, wsbase, w, chunk, end_of, copy_back, h_hist, hist_cap,
                       h_iters, st, ls.it, ls.nh, sr);
}

}  // namespace

// ===========================================================================
// Public entry points
// ===========================================================================
extern "C" {

cmf_status cmf_default_params(int algo, int L, cmf_params* p) {
    if (!p || algo < CMF_PADMM || algo > CMF_CP || L < 2) return CMF_EINVAL;
    memset(p, 0, sizeof(*p));
    p->algo = algo;
    p->storage = CMF_F32;
    p->impl = CMF_FUSED;
    p->aniso = 0;
    p->sweeps = 1;
    p->max_iter = 10000;
    p->check_every = 10;
    p->warm_start = 0;
    p->use_graph = 1;
    p->c = 0.3;
    p->a = 8.0;
    p->a1 = 2.0;
    p->a2 = 2.0 * L;
    p->rho = 1.9;
    p->r = 1.618;
    p->sigma = L == 2 ? 0.2 : 5.0;
    p->tau = L == 2 ? 1.0 : 0.4;
    if (algo == CMF_CP) {  // ALG1 (Sec. 4): sigma = 0.4, tau = 1 / (||K*K|| bound x sigma)
        p->sigma = 0.4;
        p->tau = 1.0 / ((L == 2 ? 10.0 : 9.0 + L) * 0.4);
    }
    p->tol_gap = 1e-4;
    return CMF_OK;
}

const char* cmf_status_str(cmf_status s) {
    switch (s) {
        case CMF_OK: return "ok";
        case CMF_EINVAL: return "invalid argument";
        case CMF_ENOMEM: return "workspace too small";
        case CMF_ECUDA: return "CUDA error";
        case CMF_ETIMEOUT: return "device wait timed out";
        case CMF_NOT_CONVERGED: return "not converged (max_iter reached)";
    }
    return "unknown status";
}

size_t cmf_workspace_bytes(int H, int W, int L, int pitch, const cmf_params* p) {
    if (!p || check_grid(H, W, pitch) != CMF_OK || L < 2 || L > 64) return 0;
    const size_t potts = ws_layout(H, W, L, pitch, *p, true).total;
    if (L > 2) return potts;
    const size_t binary = ws_layout(H, W, 2, pitch, *p, false).total;
    return binary > potts ? binary : potts;  // L = 2 serves both models
}

cmf_status cmf_init_binary(const float* d_Cs, const float* d_Ct, int H, int W, int pitch,
                           const cmf_params* p, float* d_u, void* d_qx, void* d_qy, void* d_ps,
                           void* d_pt, void* stream) {
    cmf_status s;
    if ((s = check_params(p, 2)) != CMF_OK) return s;
    if ((s = check_grid(H, W, pitch)) != CMF_OK) return s;
    if (!d_Cs || !d_Ct || !d_u || !d_qx || !d_qy || !d_ps || !d_pt) return CMF_EINVAL;
    BinProblem P{d_Cs, d_Ct, make_alpha(nullptr, 0.f), make_grid(H, W, pitch)};
    BinStateV st{d_u, d_qx, d_qy, d_ps, d_pt};
    CMF_CUDA_TRY(binary_init(p->storage, P, st, p->algo == CMF_RPDRQ, (float)p->tau,
                             (cudaStream_t)stream));
    return CMF_OK;
}

cmf_status cmf_iterate_binary(const float* d_Cs, const float* d_Ct, const float* d_alpha,
                              float alpha0, int H, int W, int pitch, const cmf_params* p,
                              int n_iter, float* d_u, void* d_qx, void* d_qy, void* d_ps,
                              void* d_pt, void* d_ws, size_t ws_bytes, void* stream) {
    BinaryCall c;
    cmf_status s = binary_prepare(d_Cs, d_Ct, d_alpha, alpha0, H, W, pitch, p, d_u, d_qx, d_qy,
                                  d_ps, d_pt, d_ws, ws_bytes, c);
    if (s != CMF_OK) return s;
    if (n_iter < 0) return CMF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    CMF_CUDA_TRY(cudaMemsetAsync(&((SolveCtl*)(c.wsbase + c.w.ctl))->err, 0, sizeof(int), st));
    int cur = 0;
    CMF_CUDA_TRY(binary_run(c, n_iter, cur, st));
    if (cur != 0) CMF_CUDA_TRY(copy_binary(c.user, bset(c, cur), c.P.g, c.storage, st));
    return CMF_OK;
}

cmf_status cmf_eval_binary(const float* d_Cs, const float* d_Ct, const float* d_alpha,
                           float alpha0, int H, int W, int pitch, const cmf_params* p,
                           const float* d_u, const void* d_qx, const void* d_qy,
                           const void* d_ps, const void* d_pt, double* h_out, void* d_ws,
                           size_t ws_bytes, void* stream) {
    if (!h_out) return CMF_EINVAL;
    BinaryCall c;
    cmf_status s = binary_prepare(d_Cs, d_Ct, d_alpha, alpha0, H, W, pitch, p, (float*)d_u,
                                  (void*)d_qx, (void*)d_qy, (void*)d_ps, (void*)d_pt, d_ws,
                                  ws_bytes, c);
    if (s != CMF_OK) return s;
    return binary_eval_state(c, c.user, h_out, (cudaStream_t)stream);
}

cmf_status cmf_solve_binary(const float* d_Cs, const float* d_Ct, const float* d_alpha,
                            float alpha0, int H, int W, int pitch, const cmf_params* p,
                            float* d_u, void* d_qx, void* d_qy, void* d_ps, void* d_pt,
                            double* h_hist, int hist_cap, int* h_iters, void* d_ws,
                            size_t ws_bytes, void* stream) {
    BinaryCall c;
    cmf_status s = binary_prepare(d_Cs, d_Ct, d_alpha, alpha0, H, W, pitch, p, d_u, d_qx, d_qy,
                                  d_ps, d_pt, d_ws, ws_bytes, c);
    if (s != CMF_OK) return s;
    if (hist_cap < 0) return CMF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    CMF_CUDA_TRY(cudaMemsetAsync(&((SolveCtl*)(c.wsbase + c.w.ctl))->err, 0, sizeof(int), st));
    if (!p->warm_start)
        CMF_CUDA_TRY(binary_init(c.storage, c.P, c.user, c.cfg.dr, c.cfg.dc.tau, st));
    const SolveSig sig = make_sig(0, 2, H, W, pitch, alpha0,
                                  {d_Cs, d_Ct, d_alpha, d_u, d_qx, d_qy, d_ps, d_pt, d_ws},
                                  *p);
    return solve_driver(
        p, sig, c.wsbase, c.w,
        [&](int n, int& cur, int k0, double* out) -> cmf_status {
            const EvalTail T = reduce_tail(c.wsbase, c.w);
            CMF_CUDA_TRY(cudaMemsetAsync(&T.ctl->arrive, 0, sizeof(unsigned), st));
            CMF_CUDA_TRY(binary_run(c, n, cur, st, k0, &T));
            return finish_eval(c.wsbase, c.w, out, st);
        },
        [&](int from) { return copy_binary(c.user, bset(c, from), c.P.g, c.storage, st); },
        [&](cudaStream_t s, int from, int& to, const EvalTail& T) {  // after the schedule
            to = from;
            return binary_run(c, p->check_every, to, s, p->rho_schedule_len, &T);
        },
        [&](int from) {
            int to = from;
            binary_run(c, p->check_every, to, nullptr, p->rho_schedule_len, nullptr, true);
            return to;
        },
        h_hist, hist_cap, h_iters, st);
}

cmf_status cmf_release_graphs(void) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (GraphEntry& e : *g_graphs) {
        cudaGraphExecDestroy(e.ge);
        cudaGraphDestroy(e.g);
    }
    g_graphs->clear();
    return CMF_OK;
}

cmf_status cmf_init_potts(const float* d_C, int L, int H, int W, int pitch, const cmf_params* p,
                          float* d_u, void* d_qx, void* d_qy, void* d_p, void* d_ps,
                          void* stream) {
    cmf_status s;
    if (L < 2 || L > 64) return CMF_EINVAL;
    if ((s = check_params(p, L)) != CMF_OK) return s;
    if ((s = check_grid(H, W, pitch)) != CMF_OK) return s;
    if (!d_C || !d_u || !d_qx || !d_qy || !d_p || !d_ps) return CMF_EINVAL;
    if (!aligned(d_C, p->costs == 2 ? 2 : 4)) return CMF_EINVAL;
    const PottsProblem P = potts_problem(d_C, L, nullptr, 0.f, H, W, pitch, p->costs);
    PottsStateV st{d_u, d_qx, d_qy, d_p, (float*)d_ps};
    CMF_CUDA_TRY(potts_init(p->storage, P, st, p->algo == CMF_RPDRQ, (float)p->tau,
                            (cudaStream_t)stream));
    return CMF_OK;
}

cmf_status cmf_iterate_potts(const float* d_C, int L, const float* d_alpha, float alpha0, int H,
                             int W, int pitch, const cmf_params* p, int n_iter, float* d_u,
                             void* d_qx, void* d_qy, void* d_p, void* d_ps, void* d_ws,
                             size_t ws_bytes, void* stream) {
    PottsCall c;
    cmf_status s = potts_prepare(d_C, L, d_alpha, alpha0, H, W, pitch, p, d_u, d_qx, d_qy, d_p,
                                 d_ps, d_ws, ws_bytes, c);
    if (s != CMF_OK) return s;
    if (n_iter < 0) return CMF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    CMF_CUDA_TRY(cudaMemsetAsync(c.err, 0, sizeof(int), st));
    int cur = 0;
    CMF_CUDA_TRY(potts_run(c, n_iter, cur, st));
    if (cur != 0) CMF_CUDA_TRY(copy_potts(c.user, c.ws, c.P.g, L, c.storage, st));
    return CMF_OK;
}

cmf_status cmf_eval_potts(const float* d_C, int L, const float* d_alpha, float alpha0, int H,
                          int W, int pitch, const cmf_params* p, const float* d_u,
                          const void* d_qx, const void* d_qy, const void* d_p, const void* d_ps,
                          double* h_out, void* d_ws, size_t ws_bytes, void* stream) {
    if (!h_out) return CMF_EINVAL;
    PottsCall c;
    cmf_status s = potts_prepare(d_C, L, d_alpha, alpha0, H, W, pitch, p, (float*)d_u,
                                 (void*)d_qx, (void*)d_qy, (void*)d_p, (void*)d_ps, d_ws,
                                 ws_bytes, c);
    if (s != CMF_OK) return s;
    return potts_eval_state(c, c.user, h_out, (cudaStream_t)stream);
}

// The first phase of a two-phase solve also ends when its certified gap,
// below kPhaseStallNear x phase_gap, has not fallen to kPhaseStallFactor
// times its value kPhaseStallIters iterations earlier (tested once per such
// window): the 16-bit storage's rounding floor of this instance is near (it
// rises with the step size c), and float32 storage continues from there.
constexpr int kPhaseStallIters = 200;
constexpr double kPhaseStallFactor = 0.7;
constexpr double kPhaseStallNear = 10.0;

cmf_status cmf_solve_potts(const float* d_C, int L, const float* d_alpha, float alpha0, int H,
                           int W, int pitch, const cmf_params* p, float* d_u, void* d_qx,
                           void* d_qy, void* d_p, void* d_ps, double* h_hist, int hist_cap,
                           int* h_iters, void* d_ws, size_t ws_bytes, void* stream) {
    PottsCall c;
    cmf_status s = potts_prepare(d_C, L, d_alpha, alpha0, H, W, pitch, p, d_u, d_qx, d_qy, d_p,
                                 d_ps, d_ws, ws_bytes, c);
    if (s != CMF_OK) return s;
    if (hist_cap < 0) return CMF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    CMF_CUDA_TRY(cudaMemsetAsync(c.err, 0, sizeof(int), st));
    int it0 = 0, nh0 = 0;
    if (p->phase_storage != 0) {
        // phase one: the same solve in 16-bit flow storage, in the
        // workspace's two phase sets, to the switch gap
        cmf_params q = *p;
        q.storage = p->phase_storage;
        q.tol_gap = p->phase_gap;
        q.phase_storage = 0;
        q.phase_gap = 0.0;
        const Grid G = make_grid(H, W, pitch);
        const PottsStateV A = ws_potts_state((char*)d_ws, c.w.phase, G, L, q.storage);
        const PottsStateV B =
            ws_potts_state((char*)d_ws, c.w.phase + c.w.phase_set, G, L, q.storage);
        PottsCall c1;
        s = potts_prepare(d_C, L, d_alpha, alpha0, H, W, pitch, &q, A.u, A.qx, A.qy, A.p, A.ps,
                          d_ws, ws_bytes, c1, p, &B);
        if (s != CMF_OK) return s;
        CMF_CUDA_TRY(potts_init(c1.storage, c1.P, c1.user, c1.cfg.dr, c1.cfg.dc.tau, st));
        const SolveSig sig1 = make_sig(2, L, H, W, pitch, alpha0, {d_C, d_alpha, d_ws}, q);
        int it1 = 0;
        s = solve_driver(
            &q, sig1, c1.wsbase, c1.w,
            [&](int n, int& cur, int k0, double* out) -> cmf_status {
                const EvalTail T = reduce_tail(c1.wsbase, c1.w);
                CMF_CUDA_TRY(cudaMemsetAsync(&T.ctl->arrive, 0, sizeof(unsigned), st));
                CMF_CUDA_TRY(potts_run(c1, n, cur, st, k0, &T));
                return finish_eval(c1.wsbase, c1.w, out, st);
            },
            [&](int) { return copy_potts(c1.user, c1.ws, c1.P.g, L, c1.storage, st); },
            [&](cudaStream_t s2, int from, int& to, const EvalTail& T) {
                to = from;
                return potts_run(c1, q.check_every, to, s2, 0, &T);
            },
            [&](int from) {
                int to = from;
                potts_run(c1, q.check_every, to, nullptr, 0, nullptr, true);
                return to;
            },
            h_hist, hist_cap, &it1, st, 0, 0, StallRule{kPhaseStallIters, kPhaseStallFactor,
                                                        kPhaseStallNear * q.tol_gap});
        if (s != CMF_OK && s != CMF_NOT_CONVERGED) return s;
        // the switch: the 16-bit state written exactly into the caller's
        // float32 buffers; phase two continues from it
        CMF_CUDA_TRY(potts_widen(q.storage, G, L, A, c.user, st));
        it0 = it1;
        nh0 = it1 / p->check_every;
        if (it0 >= p->max_iter) {
            CMF_CUDA_TRY(cudaStreamSynchronize(st));
            if (h_iters) *h_iters = it0;
            return CMF_NOT_CONVERGED;
        }
    } else if (!p->warm_start) {
        CMF_CUDA_TRY(potts_init(c.storage, c.P, c.user, c.cfg.dr, c.cfg.dc.tau, st));
    }
    const SolveSig sig = make_sig(1, L, H, W, pitch, alpha0,
                                  {d_C, d_alpha, d_u, d_qx, d_qy, d_p, d_ps, d_ws}, *p);
    return solve_driver(
        p, sig, c.wsbase, c.w,
        [&](int n, int& cur, int k0, double* out) -> cmf_status {
            const EvalTail T = reduce_tail(c.wsbase, c.w);
            CMF_CUDA_TRY(cudaMemsetAsync(&T.ctl->arrive, 0, sizeof(unsigned), st));
            CMF_CUDA_TRY(potts_run(c, n, cur, st, k0, &T));
            return finish_eval(c.wsbase, c.w, out, st);
        },
        [&](int) { return copy_potts(c.user, c.ws, c.P.g, L, c.storage, st); },
        [&](cudaStream_t s, int from, int& to, const EvalTail& T) {  // after the schedule
            to = from;
            return potts_run(c, p->check_every, to, s, p->rho_schedule_len, &T);
        },
        [&](int from) {
            int to = from;
            potts_run(c, p->check_every, to, nullptr, p->rho_schedule_len, nullptr, true);
            return to;
        },
        h_hist, hist_cap, h_iters, st, it0, nh0);
}

}  // extern "C"

// ===========================================================================
// Autotuner: time to the gap for each candidate launch configuration
// ===========================================================================
namespace {

// Candidate list for a parameter set: kernel variants of the fused ADMM path
// and sRBGS sweep counts of the fused rPDRQ path.
std::vector<cmf_params> tune_candidates(const cmf_params& p, bool binary) {
    std::vector<cmf_params> out;
    const bool fused = p.impl == CMF_FUSED;
    const bool dr = p.algo == CMF_RPDRQ;
    std::vector<int> variants = {p.variant};
    std::vector<int> sweeps = {p.sweeps};
    if (fused && !dr) variants = binary ? std::vector<int>{1, 2, 4, 8, 16, 32}
                                        : std::vector<int>{1, 2, 8, 16, 32};
    if (fused && dr) sweeps = {1, 2, 3};
    for (int v : variants)
        for (int s : sweeps) {
            cmf_params q = p;
            q.variant = v;
            q.sweeps = s;
            q.warm_start = 0;
            out.push_back(q);
        }
    // the ADMM step size (tune_step): larger c with the given variant
    const bool admm = p.algo == CMF_PADMM || p.algo == CMF_RPADMM_FG ||
                      p.algo == CMF_RPADMM_EB || p.algo == CMF_TY;
    if (p.tune_step == 1 && admm)
        for (double f : {2.0, 4.0, 8.0}) {
            cmf_params q = p;
            q.c = p.c * f;
            q.warm_start = 0;
            out.push_back(q);
        }
    // two-phase solves (tune_step): each step size also with the switch left
    // to the first phase's stall test alone (phase_gap 1.5 tol_gap)
    const double stall_only = 1.5 * p.tol_gap;
    if (p.tune_step == 1 && admm && p.phase_storage != 0 && stall_only < p.phase_gap)
        for (double f : {1.0, 2.0, 4.0, 8.0}) {
            cmf_params q = p;
            q.c = p.c * f;
            q.phase_gap = stall_only;
            q.warm_start = 0;
            out.push_back(q);
        }
    return out;
}

template <typename Solve>
cmf_status tune_loop(const cmf_params* p, bool binary, Solve solve, cmf_params* best,
                     double* h_best_ms, cudaStream_t st) {
    if (!p || !best) return CMF_EINVAL;
    cudaEvent_t e0, e1;
    CMF_CUDA_TRY(cudaEventCreate(&e0));
    CMF_CUDA_TRY(cudaEventCreate(&e1));
    double best_ms = 1e300;
    bool found = false;
    cmf_status last = CMF_EINVAL;
    for (const cmf_params& q : tune_candidates(*p, binary)) {
        cmf_status s = solve(q);  // warm-up (and validity check)
        last = s;
        if (s != CMF_OK) continue;
        double ms_min = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, st);
            s = solve(q);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (s == CMF_OK && ms < ms_min) ms_min = ms;
        }
        if (ms_min < best_ms) {
            best_ms = ms_min;
            *best = q;
            found = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!found) return last == CMF_OK ? CMF_NOT_CONVERGED : last;
    if (h_best_ms) *h_best_ms = best_ms;
    return CMF_OK;
}

}  // namespace

extern "C" cmf_status cmf_autotune_binary(const float* d_Cs, const float* d_Ct,
                                          const float* d_alpha, float alpha0, int H, int W,
                                          int pitch, const cmf_params* p, float* d_u,
                                          void* d_qx, void* d_qy, void* d_ps, void* d_pt,
                                          void* d_ws, size_t ws_bytes, cmf_params* best,
                                          double* h_best_ms, void* stream) {
    return tune_loop(
        p, true,
        [&](const cmf_params& q) {
            return cmf_solve_binary(d_Cs, d_Ct, d_alpha, alpha0, H, W, pitch, &q, d_u, d_qx,
                                    d_qy, d_ps, d_pt, nullptr, 0, nullptr, d_ws, ws_bytes,
                                    stream);
        },
        best, h_best_ms, (cudaStream_t)stream);
}

extern "C" cmf_status cmf_autotune_potts(const float* d_C, int L, const float* d_alpha,
                                         float alpha0, int H, int W, int pitch,
                                         const cmf_params* p, float* d_u, void* d_qx,
                                         void* d_qy, void* d_p, void* d_ps, void* d_ws,
                                         size_t ws_bytes, cmf_params* best, double* h_best_ms,
                                         void* stream) {
    return tune_loop(
        p, false,
        [&](const cmf_params& q) {
            return cmf_solve_potts(d_C, L, d_alpha, alpha0, H, W, pitch, &q, d_u, d_qx, d_qy,
                                   d_p, d_ps, nullptr, 0, nullptr, d_ws, ws_bytes, stream);
        },
        best, h_best_ms, (cudaStream_t)stream);
}
