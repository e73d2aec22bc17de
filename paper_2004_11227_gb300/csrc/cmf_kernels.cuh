// Internal interface between the C-ABI layer (cmf_api.cu) and the kernel
// translation units.  Not installed; not part of the public ABI.
#pragma once

#include <cuda.h>

#include "cmf_common.cuh"

namespace cmf {

constexpr int EVAL_ROWS = 4;  // rows per thread in the certificate kernels

// Read-only problem data of the binary model.
struct BinProblem {
    const float* Cs;
    const float* Ct;
    Alpha alpha;
    Grid g;
};

// Binary state planes with a typed flow storage.
template <typename S>
struct BinState {
    float* u;
    S* qx;
    S* qy;
    S* ps;
    S* pt;
};

// Type-erased binary state (what the host layer carries around).
struct BinStateV {
    float* u;
    void* qx;
    void* qy;
    void* ps;
    void* pt;
    template <typename S>
    __host__ __device__ BinState<S> as() const {
        return BinState<S>{u, (S*)qx, (S*)qy, (S*)ps, (S*)pt};
    }
};

// Potts problem data: L float32 cost planes at C; or (lev != NULL) one image
// plane I at C and L levels with C_i(x) = (I(x) - lev[i])^2 computed where it
// is read; or (C16 != NULL) L float16 cost planes at C16 (C then holds the
// same address, never read as float32).
struct PottsProblem {
    const float* C;
    int L;
    Alpha alpha;
    Grid g;
    const float* lev;
    const __half* C16;
};

// Cost source of a Potts problem, as the warp-strip kernels take it as a
// template parameter.
enum CostSrc { kCostF32 = 0, kCostLevels = 1, kCostF16 = 2 };
inline int cost_src(const PottsProblem& P) {
    return P.lev ? kCostLevels : (P.C16 ? kCostF16 : kCostF32);
}

// Cost of label l at plane offset k.
__device__ __forceinline__ float potts_cost(const PottsProblem& P, int l, size_t k) {
    if (P.lev) {
        const float d = __ldg(P.C + k) - __ldg(P.lev + l);
        return d * d;
    }
    if (P.C16) return __half2float(__ldg(P.C16 + (size_t)l * P.g.plane + k));
    return __ldg(P.C + (size_t)l * P.g.plane + k);
}

// Potts state: the per-label flows in the storage type S; u and the one
// p_s plane in float32.
template <typename S>
struct PottsState {
    float* u;   // L planes
    S* qx;      // L planes
    S* qy;      // L planes
    S* p;       // L planes
    float* ps;  // one plane
};

struct PottsStateV {
    float* u;
    void* qx;
    void* qy;
    void* p;
    float* ps;
    template <typename S>
    __host__ __device__ PottsState<S> as() const {
        return PottsState<S>{u, (S*)qx, (S*)qy, (S*)p, ps};
    }
};

// What one iteration launch needs besides the buffers.
struct StepConfig {
    bool dr;      // rPDRQ (else an ADMM variant)
    bool aniso;
    bool plain;   // one kernel per step (else fused)
    AdmmCoef ac;
    DrCoef dc;
};

// Block-level FP64 reduction of three accumulators; thread 0 stores the
// block's triple at out3[0..2].
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_reduce3_store(double a, double b, double c,
                                                    double* out3) {
    __shared__ double red[3][32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = a;
        red[1][tid >> 5] = b;
        red[2][tid >> 5] = c;
    }
    __syncthreads();
    if (tid < 32) {
        a = tid < nw ? red[0][tid] : 0.0;
        b = tid < nw ? red[1][tid] : 0.0;
        c = tid < nw ? red[2][tid] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_sum(c);
        if (tid == 0) {
            out3[0] = a;
            out3[1] = b;
            out3[2] = c;
        }
    }
}

// Double-float accumulator for the certificate sums: the unevaluated sum
// hi + lo of two floats, each addition made exact by Knuth's two-sum (the
// rounding error of hi goes to lo), about 44 significant bits.  GB300 runs
// FP64 arithmetic and conversions at a small fraction of its FP32 rate, so
// per-pixel terms (float32) are summed this way per lane and per warp and
// turn into FP64 once per warp; warps and blocks are summed in FP64.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void df_add(DF& a, float x) {
    const float s = a.hi + x;
    const float v = s - a.hi;
    const float err = (a.hi - (s - v)) + (x - v);
    a.hi = s;
    a.lo += err;
}

__device__ __forceinline__ void df_add(DF& a, const DF& b) {
    const float s = a.hi + b.hi;
    const float v = s - a.hi;
    const float err = (a.hi - (s - v)) + (b.hi - v);
    a.hi = s;
    a.lo = a.lo + b.lo + err;
}

__device__ __forceinline__ DF df_warp_sum(DF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF b;
        b.hi = __shfl_down_sync(0xffffffffu, a.hi, o);
        b.lo = __shfl_down_sync(0xffffffffu, a.lo, o);
        df_add(a, b);
    }
    return a;
}

__device__ __forceinline__ double df_value(const DF& a) { return (double)a.hi + (double)a.lo; }

// Block-level reduction of three double-float accumulators: per-warp sums in
// double-float, then FP64 across warps in a fixed order; thread 0 stores the
// block's triple at out3[0..2].
__device__ __forceinline__ void block_reduce3_store_df(DF a, DF b, DF c, double* out3) {
    __shared__ double red_df[3][32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y) >> 5;
    a = df_warp_sum(a);
    b = df_warp_sum(b);
    c = df_warp_sum(c);
    if ((tid & 31) == 0) {
        red_df[0][tid >> 5] = df_value(a);
        red_df[1][tid >> 5] = df_value(b);
        red_df[2][tid >> 5] = df_value(c);
    }
    __syncthreads();
    if (tid == 0) {
        double x = 0.0, y = 0.0, z = 0.0;
        for (int w = 0; w < nw; ++w) {
            x += red_df[0][w];
            y += red_df[1][w];
            z += red_df[2][w];
        }
        out3[0] = x;
        out3[1] = y;
        out3[2] = z;
    }
}

// Value a kernel stores in the workspace error word when a bounded wait runs
// out (a distinctive value, so an uninitialised workspace is not mistaken for
// a report).
constexpr int kErrWaitTimeout = 0x7E57AB1E;

// Control block in the workspace: the device-driven solve loop's counters,
// the sticky error word that kernels with bounded waits set on a timeout, and
// the arrival counter of certificate launches.
struct SolveCtl {
    int it;               // iterations done
    int checks;           // certificate evaluations done
    int stop;             // 0 running, 1 converged, 2 iteration cap, 3 device wait timed out
    int err;              // kErrWaitTimeout: a bounded device-side wait ran out
    int where;            // buffer set holding the state when the loop stopped (1 = workspace)
    unsigned int arrive;  // blocks of the current certificate launch done (0 between launches)
    double gref;          // gap at the last stall-test check (first phase of a two-phase solve)
};
static_assert(sizeof(SolveCtl) <= 64, "the workspace reserves 64 bytes for SolveCtl");

// One thread: turn the reduced (E, D, res^2) into a history row and decide
// whether the loop goes on.  The state it certified is in buffer set `where`.
// set_h: 1 = h is the loop's condition, 2 = h is the condition of the second
// half of a two-chunk loop body, 0 = leave the conditions to a later kernel.
// stall > 0 (the first phase of a two-phase solve): every `stall` checks
// the gap is compared with its value `stall` checks earlier, and the loop
// also stops, as converged, when it is below stall_near and above stall_f
// times that value (the storage's rounding floor is reached).
__device__ __forceinline__ void solve_decide(const double* scal, SolveCtl* ctl, double* hist,
                                             int hist_rows, int K, int max_iter, double tol,
                                             cudaGraphConditionalHandle h, int set_h,
                                             int where, int stall, double stall_f,
                                             double stall_near) {
    const double E = scal[0], D = scal[1], R = scal[2];
    const double gap = (E - D) / (fabs(E) > 1e-30 ? fabs(E) : 1e-30);
    const int it = ctl->it + K;
    const int n = ctl->checks;
    ctl->it = it;
    if (n < hist_rows) {
        double* row = hist + 5 * (size_t)n;
        row[0] = it;
        row[1] = E;
        row[2] = D;
        row[3] = gap;
        row[4] = sqrt(R > 0.0 ? R : 0.0);
    }
    ctl->checks = n + 1;
    bool stalled = false;
    if (stall > 0 && n % stall == 0) {
        stalled = n > 0 && gap < stall_near && gap > stall_f * ctl->gref;
        ctl->gref = gap;
    }
    const bool converged = gap <= tol || stalled;
    const bool failed = ctl->err == kErrWaitTimeout;
    const bool go = !converged && !failed && it + K <= max_iter;
    ctl->stop = go ? 0 : (failed ? 3 : (converged ? 1 : 2));
    if (!go) ctl->where = where;
    if (set_h) cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Optional completion of a certificate launch: the block that finishes last
// sums every block's partial triple in index order into scal (the same result
// for the same launch, whichever block is last) and, inside a device-driven
// solve loop, takes the stop decision.  ctl == nullptr: the launch only
// writes its partials.  ctl->arrive must be 0 when the launch starts; the
// last block sets it back to 0.
struct EvalTail {
    SolveCtl* ctl = nullptr;
    double* scal = nullptr;
    bool decide = false;
    double* hist = nullptr;
    int hist_rows = 0, K = 0, max_iter = 0;
    double tol = 0.0;
    cudaGraphConditionalHandle h = 0;
    int set_h = 0, where = 0;
    int stall = 0;  // see solve_decide
    double stall_f = 0.0, stall_near = 0.0;
};

// Called by every thread of every block after the block's partial triple is
// stored (by any thread); nblocks = the launch's block count.
__device__ __forceinline__ void eval_tail(const EvalTail& T, const double* partials,
                                          int nblocks) {
    if (!T.ctl) return;
    __shared__ int s_last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y;
    __syncthreads();
    if (tid == 0) {
        __threadfence();  // the block's partial, visible before its arrival
        s_last = atomicAdd(&T.ctl->arrive, 1u) == (unsigned)(nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = tid; i < nblocks; i += nt) {
        a += __ldcg(partials + 3 * (size_t)i);
        b += __ldcg(partials + 3 * (size_t)i + 1);
        c += __ldcg(partials + 3 * (size_t)i + 2);
    }
    block_reduce3_store(a, b, c, T.scal);
    if (tid == 0) {
        T.ctl->arrive = 0;
        if (T.decide)
            solve_decide(T.scal, T.ctl, T.hist, T.hist_rows, T.K, T.max_iter, T.tol, T.h,
                         T.set_h, T.where, T.stall, T.stall_f, T.stall_near);
    }
}

// --- launchers (binary) ---
cudaError_t binary_init(int storage, const BinProblem& P, const BinStateV& s, bool dr, float tau,
                        cudaStream_t st);
cudaError_t binary_step(int storage, const BinProblem& P, const BinStateV& a, const BinStateV& b,
                        const StepConfig& cfg, float* tmp, cudaStream_t st);
cudaError_t binary_eval(int storage, const BinProblem& P, const BinStateV& s, bool aniso, bool dr,
                        float tau, double* partials, cudaStream_t st,
                        const EvalTail& T = EvalTail());
int eval_blocks(int H, int W);

// --- launchers (Potts) ---
cudaError_t potts_init(int storage, const PottsProblem& P, const PottsStateV& s, bool dr,
                       float tau, cudaStream_t st);
// State set a (flows in `storage`) copied into float32 state set b.
cudaError_t potts_widen(int storage, const Grid& G, int L, const PottsStateV& a,
                        const PottsStateV& b, cudaStream_t st);
cudaError_t potts_step(int storage, const PottsProblem& P, const PottsStateV& a,
                       const PottsStateV& b, const StepConfig& cfg, float* tmp, cudaStream_t st);
cudaError_t potts_eval(int storage, const PottsProblem& P, const PottsStateV& s, bool aniso,
                       bool dr, float tau, double* partials, cudaStream_t st,
                       const EvalTail& T = EvalTail());

// One sRBGS preconditioner application as separate half-sweep launches
// (plain form): red, then (black, red) x D.sweeps.
cudaError_t halfsweeps(const Grid& G, float* u, const float* b, const DrCoef& D,
                       cudaStream_t st);

// --- warp-strip binary ADMM (cmf_binary_strip.cu) ---
bool binary_strip_eligible(const Grid& G, int storage, const float* Cs, const float* Ct,
                           const float* alpha, const BinStateV& a, const BinStateV& b);
cudaError_t binary_strip_step(int storage, const BinProblem& P, const BinStateV& a,
                              const BinStateV& b, bool aniso, const AdmmCoef& K,
                              cudaStream_t st);
// Two ADMM iterations from a into b in one launch (same result as two
// binary_strip_step launches through an intermediate state;
// cmf_binary_strip2.cu).  cert != nullptr: the launch also writes the
// certificates of b, one partial triple per block (at most
// binary_cert_max_blocks() of them) into `partials`, and finishes with
// eval_tail(*cert).
cudaError_t binary_strip2_step(int storage, const BinProblem& P, const BinStateV& a,
                               const BinStateV& b, bool aniso, const AdmmCoef& K,
                               cudaStream_t st, const EvalTail* cert = nullptr,
                               double* partials = nullptr);
int binary_cert_max_blocks();
// rPDRQ iteration a -> b with the pipelined red-black sweeps.
cudaError_t binary_dr_strip_step(int storage, const BinProblem& P, const BinStateV& a,
                                 const BinStateV& b, bool aniso, const DrCoef& D,
                                 cudaStream_t st);
// Certificates of a strip-eligible state into eval_blocks(H, W) partials.
cudaError_t binary_eval_strip(int storage, const BinProblem& P, const BinStateV& s, bool aniso,
                              bool dr, float tau, double* partials, cudaStream_t st,
                              const EvalTail& T);

// --- warp-strip Potts ADMM (cmf_potts_strip.cu) ---
// Eligible: even W and pitch, H * pitch within int, pair-aligned planes.
// odd_width_ok: the ADMM items of a batch also take odd widths (their last
// pair is masked; the pitch must leave room for the padding column).
bool potts_strip_eligible(const Grid& G, int storage, const float* C, const float* alpha,
                          const PottsStateV& a, const PottsStateV& b,
                          bool odd_width_ok = false);
// One iteration a -> b.  Reads u_i = a.u_i + cu_in * a.p_s; writes
// w_i = u_i^{k+1} - cu * p_s^{k+1} into b.u (see potts_strip_finalize).
cudaError_t potts_strip_step(int storage, const PottsProblem& P, const PottsStateV& a,
                             const PottsStateV& b, bool aniso, const AdmmCoef& K, float cu_in,
                             cudaStream_t st);
// Certificates of a strip-eligible state into eval_blocks(H, W) partials.
cudaError_t potts_eval_strip(int storage, const PottsProblem& P, const PottsStateV& s,
                             bool aniso, bool dr, float tau, double* partials, cudaStream_t st,
                             const EvalTail& T);
// rPDRQ iteration a -> b with the pipelined red-black sweeps (all labels).
// U_in: sum_i u_i of state a (a plane), or null to sum it from a's u planes;
// U_out: receives sum_i u_i of state b (the next launch's U_in), or null.
cudaError_t potts_dr_strip_step(int storage, const PottsProblem& P, const PottsStateV& a,
                                const PottsStateV& b, bool aniso, const DrCoef& D,
                                const float* U_in, float* U_out, cudaStream_t st);
// s.u_i += cu * s.p_s on every label (w back to u).
cudaError_t potts_strip_finalize(int storage, const PottsProblem& P, const PottsStateV& s,
                                 float cu, cudaStream_t st);

// --- TMA-staged Potts ADMM (cmf_potts_tma.cu) ---
struct PottsTmaMaps {
    CUtensorMap qx, qy, p, u, ps;
    int ty;  // output rows per tile (16 or 32)
};
bool potts_tma_eligible(const Grid& G, int storage, const PottsStateV& s);
bool potts_tma_fits(int storage, int L, int ty);  // shared memory within the block limit
// tile height (8 or 16) with the most resident warps per SM for L labels;
// ties go to 16 (less halo per output row)
int potts_tma_auto_ty(int storage, bool aniso, int L);
cudaError_t potts_tma_maps(const Grid& G, int L, int storage, const PottsStateV& s, int ty,
                           PottsTmaMaps& m);
// One iteration reading the state described by src_maps, writing b; a
// bounded TMA wait that runs out sets *err.
cudaError_t potts_admm_tma_step(int storage, const PottsProblem& P, const PottsStateV& b,
                                bool aniso, const AdmmCoef& K, const PottsTmaMaps& src_maps,
                                int* err, cudaStream_t st);

// --- TMA-staged persistent binary ADMM (cmf_binary_tma.cu) ---
struct BinTmaMaps {
    CUtensorMap qx, qy, ps, pt, u;
    int ty;  // output rows per tile (8, 16 or 32)
};
bool binary_tma_eligible(const Grid& G, int storage, const BinStateV& s);
cudaError_t binary_tma_maps(const Grid& G, int storage, const BinStateV& s, int ty,
                            BinTmaMaps& m);
cudaError_t binary_admm_tma_step(int storage, const BinProblem& P, const BinStateV& b,
                                 bool aniso, const AdmmCoef& K, const BinTmaMaps& src_maps,
                                 int* err, cudaStream_t st);

// --- batched solve (cmf_batch.cu) ---
// One instance of a batch, as the batch kernels see it (device memory).
struct BatchDesc {
    int model;       // 0 binary, 1 Potts
    int active;      // 1 while the instance still iterates
    int ntx;         // 32-wide tile columns
    int tile_base;   // first entry of this instance in its model's iteration tile table
    int ev_tab;      // first entry in its model's certificate tile table
    int ev_base;     // first certificate partial of this instance
    int ev_count;    // certificate tiles of this instance
    int iters, status;
    double energy, dual, gap, res;
    BinProblem bp;
    BinStateV bu, bw;      // caller's and workspace state (binary)
    PottsProblem pp;
    PottsStateV pu, pw;    // caller's and workspace state (Potts)
    AdmmCoef ak;           // coefficients for this instance's L
    DrCoef dk;
    int sp_nstrips;        // Potts by warp strips: strips of the grid (0: tiles)
    int sp_rows;           // band height of its strip items
};

// parity 0: caller's buffers -> workspace; 1: workspace -> caller's buffers
cudaError_t batch_binary_step(int storage, bool aniso, bool dr, int sweeps,
                              const BatchDesc* desc, const int* tile_inst, int ntiles,
                              int parity, cudaStream_t st);
cudaError_t batch_potts_step(int storage, bool aniso, bool dr, int sweeps, int rows, int maxL,
                             const BatchDesc* desc, const int* tile_inst, int ntiles,
                             int parity, cudaStream_t st);
// Potts instances of a batch by warp strips: one launch over the (instance,
// item) table (items of retired instances are skipped); first: the chunk's
// first iteration (reads u itself, later ones the w form).  The finalize
// launch turns w back into u on the same items.
cudaError_t batch_potts_strip_step(int storage, bool aniso, bool odd_width, const BatchDesc* desc,
                                   const int2* items, int nitems, int parity, int first,
                                   cudaStream_t st);
cudaError_t batch_potts_strip_finalize(const BatchDesc* desc, const int2* items, int nitems,
                                       cudaStream_t st);
int potts_strip_max_rows();  // band rows the strip kernels take at most

cudaError_t batch_binary_eval(int storage, bool aniso, bool dr, float tau,
                              const BatchDesc* desc, const int* tile_inst, int ntiles,
                              double* partials, cudaStream_t st);
cudaError_t batch_potts_eval(int storage, bool aniso, bool dr, float tau,
                             const BatchDesc* desc, const int* tile_inst, int ntiles,
                             double* partials, cudaStream_t st);

// --- reductions ---
// Sum n partial triples in a fixed order into out[0..2] (one block).
cudaError_t reduce_partials(const double* partials, int n, double* out, cudaStream_t st);

}  // namespace cmf
