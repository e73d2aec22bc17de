// Batched solve: many binary and Potts instances of uneven size and label
// count advanced together inside one CUDA graph (conditional WHILE node), with
// per-instance convergence masks.
//
// Every iteration launches one kernel over the tiles of all binary instances,
// one over the tiles of the Potts instances that run on tiles (odd widths,
// rPDRQ) and one over the warp-strip items of the other Potts instances; a
// block (tiles) or warp (strip items) maps its work to an instance through a
// device table and skips it when that instance has converged.  Every
// check_every iterations the strip instances' multipliers are turned back from
// the w form into u, the certificates of all instances are computed tile by
// tile, reduced per instance in a fixed order, and one decide kernel retires
// converged instances and sets the loop condition.
#include <math.h>
#include <string.h>

#include <vector>

#include "cmf_kernels.cuh"

namespace cmf {

namespace {

constexpr size_t kAl = 256;
inline size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }

struct BatchLayout {
    size_t desc, tiles, items, partials, scal, ctl, states, total;
    int n_bin_tiles, n_potts_tiles, n_bin_ev, n_potts_ev, potts_rows, max_l, n_strip_items;
};

// Whether a Potts instance of a batch runs by warp strips (the ADMM family,
// even pitch with room for a padding column when the width is odd,
// pair-aligned buffers; the workspace set is aligned anyway), and its strip
// and band counts.
bool batch_strip(const cmf_instance& in, const cmf_params& p) {
    if (in.model != 1 || p.algo == CMF_RPDRQ) return false;
    const Grid G{in.H, in.W, in.pitch, (size_t)in.H * (size_t)in.pitch};
    const PottsStateV s{in.d_u, in.d_qx, in.d_qy, in.d_p, (float*)in.d_ps};
    return potts_strip_eligible(G, p.storage, in.d_cost, in.d_alpha, s, s, true);
}
int strip_count(const cmf_instance& in) { return (in.W + 59) / 60; }
// band height of the strip items (params.batch_rows, 0: the kernels' maximum)
int strip_rows(const cmf_params& p) {
    return p.batch_rows > 0 ? p.batch_rows : potts_strip_max_rows();
}
int strip_items(const cmf_instance& in, const cmf_params& p) {
    const int R = strip_rows(p);
    return strip_count(in) * ((in.H + R - 1) / R);
}

int potts_rows_for(int maxL) { return maxL <= 8 ? 4 : (maxL <= 16 ? 2 : 1); }

size_t state_bytes(const cmf_instance& in, int storage) {
    const size_t plane = (size_t)in.H * (size_t)in.pitch;
    const size_t es = dtype_size(storage);
    if (in.model == 0) return al(plane * 4) + 4 * al(plane * es);
    return al(plane * 4 * in.L) + 3 * al(plane * es * in.L) + al(plane * 4);  // p_s float32
}

BatchLayout batch_layout(const cmf_instance* inst, int n, const cmf_params& p) {
    BatchLayout b{};
    int maxL = 2;
    for (int i = 0; i < n; ++i)
        if (inst[i].model == 1 && inst[i].L > maxL) maxL = inst[i].L;
    b.max_l = maxL;
    // Potts tile height: 32 rows for rPDRQ, else the fused ADMM kernel's
    // height for the largest L (its shared memory grows with L)
    b.potts_rows = p.algo == CMF_RPDRQ ? 4 : potts_rows_for(maxL);
    for (int i = 0; i < n; ++i) {
        const cmf_instance& in = inst[i];
        const int ntx = (in.W + 31) / 32;
        const int ev = ntx * ((in.H + 31) / 32);
        if (in.model == 0) {
            b.n_bin_tiles += ntx * ((in.H + 31) / 32);
            b.n_bin_ev += ev;
        } else {
            const int ty = 8 * b.potts_rows;
            if (batch_strip(in, p))
                b.n_strip_items += strip_items(in, p);
            else
                b.n_potts_tiles += ntx * ((in.H + ty - 1) / ty);
            b.n_potts_ev += ev;
        }
    }
    size_t off = 0;
    b.desc = off;
    off += al(sizeof(BatchDesc) * (size_t)n);
    b.tiles = off;
    off += al(sizeof(int) * (size_t)(b.n_bin_tiles + b.n_potts_tiles + b.n_bin_ev + b.n_potts_ev + 4));
    b.items = off;
    off += al(sizeof(int2) * (size_t)(b.n_strip_items + 1));
    b.partials = off;
    off += al(sizeof(double) * 3 * (size_t)(b.n_bin_ev + b.n_potts_ev + 1));
    b.scal = off;
    off += al(sizeof(double) * 3 * (size_t)n);
    b.ctl = off;
    off += al(64);
    b.states = off;
    for (int i = 0; i < n; ++i) off += state_bytes(inst[i], p.storage);
    b.total = off;
    return b;
}

struct BatchCtl {
    int it;
    int stop;
};

__global__ void k_batch_reset(BatchDesc* desc, int n, BatchCtl* ctl) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        desc[i].active = 1;
        desc[i].iters = 0;
        desc[i].status = CMF_NOT_CONVERGED;
    }
    if (threadIdx.x == 0) {
        ctl->it = 0;
        ctl->stop = 0;
    }
}

// One block per instance: sum its certificate partials in index order.
__global__ void k_batch_reduce(const BatchDesc* desc, const double* partials, double* scal) {
    const BatchDesc& D = desc[blockIdx.x];
    if (!D.active) return;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int t = threadIdx.x; t < D.ev_count; t += 256) {
        const size_t k = 3 * (size_t)(D.ev_base + t);
        a += partials[k];
        b += partials[k + 1];
        c += partials[k + 2];
    }
    __shared__ double red[3][8];
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = b;
        red[2][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < 8; ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
            s2 += red[2][w];
        }
        scal[3 * blockIdx.x] = s0;
        scal[3 * blockIdx.x + 1] = s1;
        scal[3 * blockIdx.x + 2] = s2;
    }
}

// One block: retire converged instances, decide whether the loop runs again.
// set_h = 0: a host-driven loop (no graph), which reads ctl->stop instead.
__global__ void k_batch_decide(BatchDesc* desc, int n, const double* scal, BatchCtl* ctl, int K,
                               int max_iter, double tol, cudaGraphConditionalHandle h,
                               int set_h) {
    const int it = ctl->it + K;
    int any = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        BatchDesc& D = desc[i];
        if (!D.active) continue;
        const double E = scal[3 * i], Dv = scal[3 * i + 1], R = scal[3 * i + 2];
        const double gap = (E - Dv) / (fabs(E) > 1e-30 ? fabs(E) : 1e-30);
        D.iters = it;
        D.energy = E;
        D.dual = Dv;
        D.gap = gap;
        D.res = sqrt(R > 0.0 ? R : 0.0);
        if (gap <= tol) {
            D.active = 0;
            D.status = CMF_OK;
        } else if (it + K > max_iter) {
            D.active = 0;
            D.status = CMF_NOT_CONVERGED;
        } else {
            any = 1;
        }
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        ctl->it = it;
        ctl->stop = any ? 0 : 1;
        if (set_h) cudaGraphSetConditional(h, any ? 1u : 0u);
    }
}

cmf_status check_instance(const cmf_instance& in, const cmf_params& p) {
    if (in.model != 0 && in.model != 1) return CMF_EINVAL;
    if (in.model == 0 && in.L != 2) return CMF_EINVAL;
    if (in.model == 1 && (in.L < 2 || in.L > 64)) return CMF_EINVAL;
    if (in.H < 1 || in.W < 1 || in.pitch < in.W) return CMF_EINVAL;
    if (!in.d_cost || !in.d_u || !in.d_qx || !in.d_qy || !in.d_p || !in.d_ps) return CMF_EINVAL;
    if (!in.d_alpha && !(in.alpha0 >= 0.0f && isfinite(in.alpha0))) return CMF_EINVAL;
    const size_t es = dtype_size(p.storage);
    auto ok = [](const void* q, size_t a) { return ((uintptr_t)q % a) == 0; };
    if (!ok(in.d_cost, 4) || !ok(in.d_u, 4) || (in.d_alpha && !ok(in.d_alpha, 4))) return CMF_EINVAL;
    // the Potts p_s plane is float32 for every flow storage
    const size_t es_ps = in.model == 1 ? 4 : es;
    if (!ok(in.d_qx, es) || !ok(in.d_qy, es) || !ok(in.d_p, es) || !ok(in.d_ps, es_ps))
        return CMF_EINVAL;
    return CMF_OK;
}

cmf_status check_batch_params(const cmf_params* p) {
    if (!p) return CMF_EINVAL;
    if (p->algo < CMF_PADMM || p->algo > CMF_CP) return CMF_EINVAL;
    if (p->costs != 0) return CMF_EINVAL;  // batches take cost planes
    if (p->phase_storage != 0) return CMF_EINVAL;  // two-phase solves: single Potts solves only
    if (p->rho_schedule_len != 0) return CMF_EINVAL;  // one rho for every instance
    if (p->storage < CMF_F32 || p->storage > CMF_BF16) return CMF_EINVAL;
    if (p->impl != CMF_FUSED) return CMF_EINVAL;  // the batch runs the fused kernels
    if (p->sweeps != 1) return CMF_EINVAL;  // batched rPDRQ runs one sRBGS sweep
    if (!(p->c > 0) || !(p->a > 0) || !(p->a1 > 0) || !(p->a2 >= 0)) return CMF_EINVAL;
    if (!(p->rho > 0) || !(p->rho < 2) || !(p->r > 0) || !(p->sigma > 0) || !(p->tau > 0))
        return CMF_EINVAL;
    // whole chunks, and an even chunk so every chunk ends in the callers' buffers
    if (p->check_every < 2 || (p->check_every & 1) || p->max_iter < p->check_every ||
        p->max_iter % p->check_every)
        return CMF_EINVAL;
    if (!(p->tol_gap >= 0)) return CMF_EINVAL;
    if (p->batch_rows != 0 && (p->batch_rows < 8 || p->batch_rows > potts_strip_max_rows()))
        return CMF_EINVAL;
    return CMF_OK;
}

}  // namespace
}  // namespace cmf

using namespace cmf;

extern "C" size_t cmf_batch_workspace_bytes(const cmf_instance* inst, int n, const cmf_params* p) {
    if (!inst || n < 1 || !p || check_batch_params(p) != CMF_OK) return 0;
    for (int i = 0; i < n; ++i)
        if (check_instance(inst[i], *p) != CMF_OK) return 0;
    return batch_layout(inst, n, *p).total;
}

extern "C" cmf_status cmf_solve_batch(cmf_instance* inst, int n, const cmf_params* p,
                                      void* d_ws, size_t ws_bytes, void* stream) {
    cmf_status s;
    if (!inst || n < 1 || !d_ws) return CMF_EINVAL;
    if ((s = check_batch_params(p)) != CMF_OK) return s;
    for (int i = 0; i < n; ++i)
        if ((s = check_instance(inst[i], *p)) != CMF_OK) return s;
    if ((uintptr_t)d_ws % kAl) return CMF_EINVAL;
    const BatchLayout B = batch_layout(inst, n, *p);
    if (ws_bytes < B.total) return CMF_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)d_ws;
    const bool dr = p->algo == CMF_RPDRQ;
    const bool aniso = p->aniso != 0;
    const size_t es = dtype_size(p->storage);

    // descriptors and tile tables
    std::vector<BatchDesc> desc(n);
    std::vector<int> tb, tp, eb, ep;
    // (instance, strip item) of the strip-eligible Potts instances, even and
    // odd widths apart (the odd ones run the kernel with the last-pair masks)
    std::vector<int2> sitems, oitems;
    char* sbase = ws + B.states;
    const int pty = 8 * B.potts_rows;
    for (int i = 0; i < n; ++i) {
        const cmf_instance& in = inst[i];
        BatchDesc& D = desc[i];
        memset(&D, 0, sizeof(D));
        D.model = in.model;
        const Grid G{in.H, in.W, in.pitch, (size_t)in.H * (size_t)in.pitch};
        const size_t plane = G.plane;
        const int ntx = (in.W + 31) / 32;
        D.ntx = ntx;
        D.ev_base = (int)(in.model == 0 ? eb.size() : B.n_bin_ev + ep.size());
        D.ev_count = ntx * ((in.H + 31) / 32);
        const Alpha A{in.d_alpha, in.alpha0};
        // Thm 2 needs a2 >= 2L: each Potts instance uses max(p->a2, 2L).
        // ALG1 needs sigma tau ||K*K|| <= 1: each instance uses
        // min(p->tau, 1 / (bound x sigma)), the bound of cmf_default_params
        // for its L (10 binary, 9 + L Potts)
        cmf_params pi = *p;
        if (in.model == 1 && pi.a2 < 2.0 * in.L) pi.a2 = 2.0 * in.L;
        if (p->algo == CMF_CP) {
            const double bound = in.model == 0 ? 10.0 : 9.0 + in.L;
            const double tmax = 1.0 / (bound * pi.sigma);
            if (pi.tau > tmax) pi.tau = tmax;
        }
        D.ak = make_admm_coef(pi, in.model == 0 ? 2 : in.L);
        D.dk = make_dr_coef(pi, in.model == 0 ? 2 : in.L, in.model == 1);
        if (in.model == 0) {
            D.bp = BinProblem{in.d_cost, in.d_cost + plane, A, G};
            D.bu = BinStateV{in.d_u, in.d_qx, in.d_qy, in.d_ps, in.d_p};
            char* b = sbase;
            D.bw.u = (float*)b;
            b += al(plane * 4);
            D.bw.qx = b;
            b += al(plane * es);
            D.bw.qy = b;
            b += al(plane * es);
            D.bw.ps = b;
            b += al(plane * es);
            D.bw.pt = b;
            D.tile_base = (int)tb.size();
            D.ev_tab = (int)eb.size();
            for (int t = 0; t < ntx * ((in.H + 31) / 32); ++t) tb.push_back(i);
            for (int t = 0; t < D.ev_count; ++t) eb.push_back(i);
        } else {
            D.pp = PottsProblem{in.d_cost, in.L, A, G, nullptr};
            D.pu = PottsStateV{in.d_u, in.d_qx, in.d_qy, in.d_p, (float*)in.d_ps};
            char* b = sbase;
            D.pw.u = (float*)b;
            b += al(plane * 4 * in.L);
            D.pw.qx = b;
            b += al(plane * es * in.L);
            D.pw.qy = b;
            b += al(plane * es * in.L);
            D.pw.p = b;
            b += al(plane * es * in.L);
            D.pw.ps = (float*)b;
            D.tile_base = (int)tp.size();
            D.ev_tab = (int)ep.size();
            if (batch_strip(in, *p)) {
                D.sp_nstrips = strip_count(in);
                D.sp_rows = strip_rows(*p);
                std::vector<int2>& dst = in.W % 2 ? oitems : sitems;
                for (int t = 0; t < strip_items(in, *p); ++t) dst.push_back(make_int2(i, t));
            } else {
                for (int t = 0; t < ntx * ((in.H + pty - 1) / pty); ++t) tp.push_back(i);
            }
            for (int t = 0; t < D.ev_count; ++t) ep.push_back(i);
        }
        sbase += state_bytes(in, p->storage);
    }
    int* tables = (int*)(ws + B.tiles);
    int* d_tb = tables;
    int* d_tp = d_tb + tb.size();
    int* d_eb = d_tp + tp.size();
    int* d_ep = d_eb + eb.size();
    std::vector<int> all;
    all.reserve(tb.size() + tp.size() + eb.size() + ep.size());
    all.insert(all.end(), tb.begin(), tb.end());
    all.insert(all.end(), tp.begin(), tp.end());
    all.insert(all.end(), eb.begin(), eb.end());
    all.insert(all.end(), ep.begin(), ep.end());
    BatchDesc* d_desc = (BatchDesc*)(ws + B.desc);
    double* partials = (double*)(ws + B.partials);
    double* scal = (double*)(ws + B.scal);
    BatchCtl* ctl = (BatchCtl*)(ws + B.ctl);
    CMF_CUDA_TRY(cudaMemcpyAsync(d_desc, desc.data(), sizeof(BatchDesc) * n,
                                 cudaMemcpyHostToDevice, st));
    if (!all.empty())
        CMF_CUDA_TRY(cudaMemcpyAsync(tables, all.data(), sizeof(int) * all.size(),
                                     cudaMemcpyHostToDevice, st));
    int2* d_items = (int2*)(ws + B.items);
    int2* d_oitems = d_items + sitems.size();
    if (!sitems.empty())
        CMF_CUDA_TRY(cudaMemcpyAsync(d_items, sitems.data(), sizeof(int2) * sitems.size(),
                                     cudaMemcpyHostToDevice, st));
    if (!oitems.empty())
        CMF_CUDA_TRY(cudaMemcpyAsync(d_oitems, oitems.data(), sizeof(int2) * oitems.size(),
                                     cudaMemcpyHostToDevice, st));
    // cold starts
    if (!p->warm_start) {
        for (int i = 0; i < n; ++i) {
            const BatchDesc& D = desc[i];
            if (D.model == 0)
                CMF_CUDA_TRY(binary_init(p->storage, D.bp, D.bu, dr, (float)p->tau, st));
            else
                CMF_CUDA_TRY(potts_init(p->storage, D.pp, D.pu, dr, (float)p->tau, st));
        }
    }
    k_batch_reset<<<1, 256, 0, st>>>(d_desc, n, ctl);
    CMF_CUDA_TRY(cudaGetLastError());

    // one chunk: check_every iterations of every active instance, the
    // certificates and the per-instance stop decision
    auto enqueue_chunk = [&](cudaStream_t s, cudaGraphConditionalHandle h,
                             int set_h) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < p->check_every && e == cudaSuccess; ++k) {
            const int parity = k & 1;
            if (!tb.empty())
                e = batch_binary_step(p->storage, aniso, dr, p->sweeps, d_desc, d_tb,
                                      (int)tb.size(), parity, s);
            if (e == cudaSuccess && !tp.empty())
                e = batch_potts_step(p->storage, aniso, dr, p->sweeps, B.potts_rows, B.max_l,
                                     d_desc, d_tp, (int)tp.size(), parity, s);
            if (e == cudaSuccess && !sitems.empty())
                e = batch_potts_strip_step(p->storage, aniso, false, d_desc, d_items,
                                           (int)sitems.size(), parity, k == 0, s);
            if (e == cudaSuccess && !oitems.empty())
                e = batch_potts_strip_step(p->storage, aniso, true, d_desc, d_oitems,
                                           (int)oitems.size(), parity, k == 0, s);
        }
        // the strip instances hold w = u - cu p_s after the chunk: back to u
        // (both tables are contiguous in the workspace)
        const int nall = (int)(sitems.size() + oitems.size());
        if (e == cudaSuccess && nall > 0)
            e = batch_potts_strip_finalize(d_desc, d_items, nall, s);
        if (e == cudaSuccess && !eb.empty())
            e = batch_binary_eval(p->storage, aniso, dr, (float)p->tau, d_desc, d_eb,
                                  (int)eb.size(), partials, s);
        if (e == cudaSuccess && !ep.empty())
            e = batch_potts_eval(p->storage, aniso, dr, (float)p->tau, d_desc, d_ep,
                                 (int)ep.size(), partials, s);
        if (e == cudaSuccess) {
            k_batch_reduce<<<n, 256, 0, s>>>(d_desc, partials, scal);
            k_batch_decide<<<1, 256, 0, s>>>(d_desc, n, scal, ctl, p->check_every, p->max_iter,
                                              p->tol_gap, h, set_h);
            e = cudaGetLastError();
        }
        return e;
    };
    auto collect = [&]() -> cmf_status {
        bool all_ok = true;
        for (int i = 0; i < n; ++i) {
            inst[i].iters = desc[i].iters;
            inst[i].status = desc[i].status;
            inst[i].energy = desc[i].energy;
            inst[i].dual = desc[i].dual;
            inst[i].gap = desc[i].gap;
            inst[i].res = desc[i].res;
            all_ok = all_ok && desc[i].status == CMF_OK;
        }
        return all_ok ? CMF_OK : CMF_NOT_CONVERGED;
    };
    if (!p->use_graph) {
        // host-driven: one chunk per round trip, the stop flag read back
        for (;;) {
            CMF_CUDA_TRY(enqueue_chunk(st, 0, 0));
            BatchCtl hc;
            CMF_CUDA_TRY(cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, st));
            CMF_CUDA_TRY(cudaStreamSynchronize(st));
            if (hc.stop) break;
        }
        CMF_CUDA_TRY(cudaMemcpyAsync(desc.data(), d_desc, sizeof(BatchDesc) * n,
                                     cudaMemcpyDeviceToHost, st));
        CMF_CUDA_TRY(cudaStreamSynchronize(st));
        return collect();
    }

    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cmf_status status = CMF_ECUDA;
    do {
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) break;
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
        if (cudaStreamBeginCaptureToGraph(cs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed) != cudaSuccess)
            break;
        const cudaError_t e = enqueue_chunk(cs, h, 1);
        cudaGraph_t captured = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
        if (e != cudaSuccess || e2 != cudaSuccess) break;
        if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) break;
        if (cudaGraphLaunch(ge, st) != cudaSuccess) break;
        if (cudaMemcpyAsync(desc.data(), d_desc, sizeof(BatchDesc) * n, cudaMemcpyDeviceToHost,
                            st) != cudaSuccess)
            break;
        if (cudaStreamSynchronize(st) != cudaSuccess) break;
        status = collect();
    } while (0);
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
    return status;
}

extern "C" cmf_status cmf_autotune_batch(cmf_instance* inst, int n, const cmf_params* p,
                                         cmf_params* best, double* h_best_ms, void* d_ws,
                                         size_t ws_bytes, void* stream) {
    if (!inst || n < 1 || !p || !best) return CMF_EINVAL;
    cmf_status s;
    if ((s = check_batch_params(p)) != CMF_OK) return s;
    bool strips = false;
    for (int i = 0; i < n; ++i) {
        if ((s = check_instance(inst[i], *p)) != CMF_OK) return s;
        strips = strips || batch_strip(inst[i], *p);
    }
    std::vector<cmf_params> cand;
    for (int f : {1, 2, 5}) {
        const int k = p->check_every * f;
        if (k > p->max_iter || p->max_iter % k) continue;
        for (int rows : {12, 16, 24}) {
            if (!strips && rows != 24) continue;
            cmf_params q = *p;
            q.check_every = k;
            q.batch_rows = rows;
            q.warm_start = 0;
            cand.push_back(q);
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    // one untimed solve first: module loading and first launches
    if (!cand.empty() && batch_layout(inst, n, cand[0]).total <= ws_bytes) {
        s = cmf_solve_batch(inst, n, &cand[0], d_ws, ws_bytes, stream);
        if (s == CMF_ECUDA || s == CMF_ETIMEOUT || s == CMF_EINVAL) return s;
    }
    cudaEvent_t e0, e1;
    CMF_CUDA_TRY(cudaEventCreate(&e0));
    CMF_CUDA_TRY(cudaEventCreate(&e1));
    double best_ms = 1e300;
    bool found = false;
    cmf_status last = CMF_NOT_CONVERGED;
    for (const cmf_params& q : cand) {
        if (batch_layout(inst, n, q).total > ws_bytes) {
            last = CMF_ENOMEM;
            continue;
        }
        cudaEventRecord(e0, st);
        s = cmf_solve_batch(inst, n, &q, d_ws, ws_bytes, stream);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (s == CMF_ECUDA || s == CMF_ETIMEOUT) {
            last = s;
            break;
        }
        if (s != CMF_OK) continue;
        if (ms < best_ms) {
            best_ms = ms;
            *best = q;
            found = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!found) return last;
    if (h_best_ms) *h_best_ms = best_ms;
    return CMF_OK;
}
