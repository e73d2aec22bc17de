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

// Potts problem data: L cost planes, or (lev != NULL) one image plane I in C
// and L levels with C_i(x) = (I(x) - lev[i])^2 computed where it is read.
struct PottsProblem {
    const float* C;
    int L;
    Alpha alpha;
    Grid g;
    const float* lev;
};

// Cost of label l at plane offset k.
__device__ __forceinline__ float potts_cost(const PottsProblem& P, int l, size_t k) {
    if (P.lev) {
        const float d = __ldg(P.C + k) - __ldg(P.lev + l);
        return d * d;
    }
    return __ldg(P.C + (size_t)l * P.g.plane + k);
}

template <typename S>
struct PottsState {
    float* u;   // L planes
    S* qx;      // L planes
    S* qy;      // L planes
    S* p;       // L planes
    S* ps;      // one plane
};

struct PottsStateV {
    float* u;
    void* qx;
    void* qy;
    void* p;
    void* ps;
    template <typename S>
    __host__ __device__ PottsState<S> as() const {
        return PottsState<S>{u, (S*)qx, (S*)qy, (S*)p, (S*)ps};
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

// --- launchers (binary) ---
cudaError_t binary_init(int storage, const BinProblem& P, const BinStateV& s, bool dr, float tau,
                        cudaStream_t st);
cudaError_t binary_step(int storage, const BinProblem& P, const BinStateV& a, const BinStateV& b,
                        const StepConfig& cfg, float* tmp, cudaStream_t st);
cudaError_t binary_eval(int storage, const BinProblem& P, const BinStateV& s, bool aniso, bool dr,
                        float tau, double* partials, cudaStream_t st);
int eval_blocks(int H, int W);

// --- launchers (Potts) ---
cudaError_t potts_init(int storage, const PottsProblem& P, const PottsStateV& s, bool dr,
                       float tau, cudaStream_t st);
cudaError_t potts_step(int storage, const PottsProblem& P, const PottsStateV& a,
                       const PottsStateV& b, const StepConfig& cfg, float* tmp, cudaStream_t st);
cudaError_t potts_eval(int storage, const PottsProblem& P, const PottsStateV& s, bool aniso,
                       bool dr, float tau, double* partials, cudaStream_t st);

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
// cmf_binary_strip2.cu).
cudaError_t binary_strip2_step(int storage, const BinProblem& P, const BinStateV& a,
                               const BinStateV& b, bool aniso, const AdmmCoef& K,
                               cudaStream_t st);
// rPDRQ iteration a -> b with the pipelined red-black sweeps.
cudaError_t binary_dr_strip_step(int storage, const BinProblem& P, const BinStateV& a,
                                 const BinStateV& b, bool aniso, const DrCoef& D,
                                 cudaStream_t st);
// Certificates of a strip-eligible state into eval_blocks(H, W) partials.
cudaError_t binary_eval_strip(int storage, const BinProblem& P, const BinStateV& s, bool aniso,
                              bool dr, float tau, double* partials, cudaStream_t st);

// --- warp-strip Potts ADMM (cmf_potts_strip.cu) ---
// Eligible: even W and pitch, H * pitch within int, pair-aligned planes.
bool potts_strip_eligible(const Grid& G, int storage, const float* C, const float* alpha,
                          const PottsStateV& a, const PottsStateV& b);
// One iteration a -> b.  Reads u_i = a.u_i + cu_in * a.p_s; writes
// w_i = u_i^{k+1} - cu * p_s^{k+1} into b.u (see potts_strip_finalize).
cudaError_t potts_strip_step(int storage, const PottsProblem& P, const PottsStateV& a,
                             const PottsStateV& b, bool aniso, const AdmmCoef& K, float cu_in,
                             cudaStream_t st);
// Certificates of a strip-eligible state into eval_blocks(H, W) partials.
cudaError_t potts_eval_strip(int storage, const PottsProblem& P, const PottsStateV& s,
                             bool aniso, bool dr, float tau, double* partials, cudaStream_t st);
// rPDRQ iteration a -> b with the pipelined red-black sweeps (all labels).
cudaError_t potts_dr_strip_step(int storage, const PottsProblem& P, const PottsStateV& a,
                                const PottsStateV& b, bool aniso, const DrCoef& D,
                                cudaStream_t st);
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
};

// parity 0: caller's buffers -> workspace; 1: workspace -> caller's buffers
cudaError_t batch_binary_step(int storage, bool aniso, bool dr, int sweeps,
                              const BatchDesc* desc, const int* tile_inst, int ntiles,
                              int parity, cudaStream_t st);
cudaError_t batch_potts_step(int storage, bool aniso, bool dr, int sweeps, int rows, int maxL,
                             const BatchDesc* desc, const int* tile_inst, int ntiles,
                             int parity, cudaStream_t st);
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
