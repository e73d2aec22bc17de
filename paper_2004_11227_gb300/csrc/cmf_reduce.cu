// Deterministic final pass of the FP64 certificate reductions, and the
// host-side coefficient bundles of the iterations.
#include "cmf_kernels.cuh"

namespace cmf {

// One block of 256 threads: thread t adds partials t, t+256, ... in index
// order, then a fixed shuffle tree combines the threads.  The result depends
// only on n and the partials, never on scheduling.
__global__ void __launch_bounds__(256) k_reduce_partials(const double* partials, int n,
                                                         double* out) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        a += partials[3 * (size_t)i + 0];
        b += partials[3 * (size_t)i + 1];
        c += partials[3 * (size_t)i + 2];
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
        out[0] = s0;
        out[1] = s1;
        out[2] = s2;
    }
}

cudaError_t reduce_partials(const double* partials, int n, double* out, cudaStream_t st) {
    k_reduce_partials<<<1, 256, 0, st>>>(partials, n, out);
    return cudaGetLastError();
}

AdmmCoef make_admm_coef(const cmf_params& p, int L) {
    const bool eb = p.algo == CMF_RPADMM_EB;
    const bool ty = p.algo == CMF_TY;
    const double rho_p = eb ? p.rho : 1.0;
    const double r = p.algo == CMF_RPADMM_FG ? p.r : 1.0;
    const double a2 = p.a2 > 0.0 ? p.a2 : 2.0 * L;
    AdmmCoef k;
    k.inv_a = (float)(1.0 / p.a);
    k.inv_c = (float)(1.0 / p.c);
    k.rho_p = (float)rho_p;
    k.rho_a1 = (float)(rho_p / p.a1);
    k.inv_a1 = (float)(1.0 / p.a1);
    k.inv_a2 = (float)(1.0 / a2);
    k.cu = (float)((eb || ty) ? p.c : r * p.c);
    k.omr = (float)(eb ? 1.0 - p.rho : 0.0);
    k.inv_L = (float)(1.0 / L);
    k.ty = ty ? 1 : 0;
    k.cp = 0;
    k.sigma = (float)p.sigma;
    k.tau = (float)p.tau;
    if (p.algo == CMF_CP) {  // g = -ubar / tau; q-step q + sigma tau grad g; u = v + tau p_s
        k.cp = 1;
        k.inv_c = (float)(1.0 / p.tau);
        k.inv_a = (float)(p.sigma * p.tau);
        k.cu = (float)p.tau;
    }
    return k;
}

DrCoef make_dr_coef(const cmf_params& p, int L, bool potts) {
    DrCoef d;
    d.sigma = (float)p.sigma;
    d.tau = (float)p.tau;
    d.rho = (float)p.rho;
    d.inv_st = (float)(1.0 / (p.sigma * p.tau));
    d.kappa = (float)(potts ? L + 1.0 : 2.0);  // T = -Lap + 2I or T_0 = -Lap + (L+1) I
    d.Lm1 = (float)(L - 1);
    d.sweeps = p.sweeps;
    return d;
}

}  // namespace cmf
