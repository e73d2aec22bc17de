// cmf_eval_binary_noalloc: the binary certificate evaluation without a
// caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they want a
// certificate: plug-ins that receive only a stream and the solver's buffers
// from a host application that owns every allocation, and real-time loops
// whose memory budget is fixed up front.  This entry point keeps its scratch
// (the per-block partial sums and the reduced scalars) in a file-scope
// __device__ array instead.  The array exists on every GPU that loads the
// library, for as long as the library stays loaded.  The call synchronises
// its stream and copies the result to the host, so it refuses to run on a
// stream that is being captured into a CUDA graph.
#include <math.h>

#include "cmf_kernels.cuh"

namespace {

// Scratch capacity: partial triples for up to kMaxBlocks certificate blocks
// (each block covers 32 x 32 pixels, so 16384 blocks cover a 4096 x 4096
// grid) plus 4 reduced scalars.  3 * 16384 + 4 doubles = 393,248 bytes.
constexpr int kMaxBlocks = 16384;
constexpr int kScratchDoubles = 3 * kMaxBlocks + 4;

static __device__ __align__(256) double g_eval_scratch[kScratchDoubles];

// Device address of g_eval_scratch on the current device.  In host code the
// name g_eval_scratch is only a host-side stand-in; kernels must be given the
// address cudaGetSymbolAddress returns.  It is looked up on every call (after
// the capture check, so never during a capture): a table cached across calls
// would keep a dead address after cudaDeviceReset reloads the module.
cudaError_t scratch_for_current_device(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_eval_scratch);
    if (e != cudaSuccess) return e;
    *out = (double*)p;
    return cudaSuccess;
}

}  // namespace

extern "C" cmf_status cmf_eval_binary_noalloc(const float* d_Cs, const float* d_Ct,
                                              const float* d_alpha, float alpha0, int H, int W,
                                              int pitch, const cmf_params* p, const float* d_u,
                                              const void* d_qx, const void* d_qy,
                                              const void* d_ps, const void* d_pt, double* h_out,
                                              void* stream) {
    using namespace cmf;
    if (!p || !h_out || !d_Cs || !d_Ct || !d_u || !d_qx || !d_qy || !d_ps || !d_pt)
        return CMF_EINVAL;
    if (H < 1 || W < 1 || pitch < W) return CMF_EINVAL;
    if (p->algo < CMF_PADMM || p->algo > CMF_CP) return CMF_EINVAL;
    if (p->storage < CMF_F32 || p->storage > CMF_BF16) return CMF_EINVAL;
    if (!(p->tau > 0)) return CMF_EINVAL;
    if (!d_alpha && !(alpha0 >= 0.0f && isfinite(alpha0))) return CMF_EINVAL;
    const int nblocks = eval_blocks(H, W);
    if (nblocks > kMaxBlocks) return CMF_EINVAL;  // grid larger than the static scratch

    cudaStream_t st = (cudaStream_t)stream;
    // the call ends with a device-to-host copy and a stream synchronisation,
    // neither of which a stream capture allows: refuse before any launch
    // (the query itself is allowed during a capture and leaves it valid)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return CMF_EINVAL;

    double* scratch = nullptr;
    CMF_CUDA_TRY(scratch_for_current_device(&scratch));
    double* partials = scratch;
    double* scal = scratch + 3 * kMaxBlocks;

    BinProblem P{d_Cs, d_Ct, Alpha{d_alpha, alpha0},
                 Grid{H, W, pitch, (size_t)H * (size_t)pitch}};
    BinStateV s{(float*)d_u, (void*)d_qx, (void*)d_qy, (void*)d_ps, (void*)d_pt};
    // every block writes its own partial triple and the final pass overwrites
    // the scalars, so nothing in the scratch has to start at zero
    CMF_CUDA_TRY(binary_eval(p->storage, P, s, p->aniso != 0, p->algo == CMF_RPDRQ,
                             (float)p->tau, partials, st));
    CMF_CUDA_TRY(reduce_partials(partials, nblocks, scal, st));
    double h[3];
    CMF_CUDA_TRY(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, st));
    CMF_CUDA_TRY(cudaStreamSynchronize(st));
    h_out[0] = h[0];
    h_out[1] = h[1];
    h_out[2] = (h[0] - h[1]) / (fabs(h[0]) > 1e-30 ? fabs(h[0]) : 1e-30);
    h_out[3] = sqrt(h[2] > 0 ? h[2] : 0.0);
    return CMF_OK;
}
