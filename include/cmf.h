/*
 * cmf.h -- C ABI of libcmf, a GB300 (sm_103a) solver for continuous max-flow
 * / min-cut image segmentation after Sun, Tai and Yuan, "Efficient ADMM and
 * splitting methods for continuous min-cut and max-flow problems".
 *
 * Problems (Sec. 2.1):
 *   binary  max sum_x p_s  s.t. |q(x)| <= alpha(x), p_s <= C_s, p_t <= C_t,
 *           div q - p_s + p_t = 0                       (Eq. two-label-mf)
 *           dual of  min_{u in [0,1]} sum (1-u) C_s + u C_t + alpha |grad u|
 *                                                       (Eq. seg:chanvese)
 *   Potts   max sum_x p_s  s.t. |q_i| <= alpha, p_i <= C_i,
 *           div q_i - p_s + p_i = 0, i = 1..L           (Eq. potts-mf)
 *           dual of the simplex-constrained relaxed Potts model
 *                                                       (Eq. relaxed-potts)
 * The multiplier u of the conservation constraint is the relaxed labelling.
 *
 * Algorithms (Sec. 3): pADMMI (Fortin-Glowinski ADMM without relaxation,
 * Sec. 4), rpADMMI (Eq. rpADMMI / Eq. multi:fg:4), rpADMMII (Eq. rpADMMII /
 * the Potts Eckstein-Bertsekas equations after Thm 2), rPDRQ (Eq.
 * iteration:quadratic:seg / Eq. pdrq:4labels) with a symmetric red-black
 * Gauss-Seidel preconditioner.
 *
 * Discretisation: unit grid spacing, forward-difference gradient that is 0 on
 * the far boundary, div = -grad^T (the scheme behind ||div^* div|| <= 8 in
 * Thm 1).
 *
 * Conventions shared by every entry point
 *  - Grids are H rows x W columns, row-major with a row stride of `pitch`
 *    elements (pitch >= W).  A "plane" is H*pitch elements; stacked planes
 *    follow each other with no gap.  Padding columns are never read or
 *    written.
 *  - Pointers named d_* are DEVICE pointers owned by the caller; the library
 *    never frees them and never allocates device memory inside a call except
 *    where stated (the CUDA graph objects of cmf_solve_*, kept for reuse, see
 *    cmf_release_graphs).  Pointers named h_* are HOST pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream-ordered: device outputs are valid once the
 *    stream has been synchronised.  Entry points that return host values
 *    (cmf_eval_*, cmf_solve_*) synchronise the stream themselves.
 *  - Errors are returned, never aborted on.  On CMF_EINVAL nothing was
 *    launched.  On CMF_ECUDA the state buffers are undefined.
 *  - Kernels that stage data with TMA wait on shared-memory barriers with a
 *    bound of about one second; a wait that runs out makes the kernel record
 *    the event in the workspace and return (the state is then undefined).
 *    cmf_solve_* report it as CMF_ETIMEOUT; after cmf_iterate_* (which does
 *    not synchronise) the next cmf_eval_* on the same workspace reports it.
 *    cmf_iterate_* and cmf_solve_* clear the record when they start.
 *  - State storage: u is always float32.  Flows (binary q, p_s, p_t; Potts
 *    q_i, p_i) are stored as cmf_params.storage (float32, float16 or
 *    bfloat16); the Potts source flow p_s, one plane shared by all labels, is
 *    always float32 (4 bytes per pixel more than 16 bits; rounded to 16 bits
 *    it alone holds the certified gap of a 16-label problem near 4e-4); all
 *    arithmetic is float32; the certificates (energies, gap, residual) sum
 *    float32 per-pixel terms in double-float (two floats kept exact by
 *    two-sum, about 44 significant bits) within a warp and in float64 above
 *    it.
 */
#ifndef CMF_H
#define CMF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CMF_OK = 0,
    CMF_EINVAL = 1,        /* bad argument: sizes, pointers, parameters       */
    CMF_ENOMEM = 2,        /* workspace smaller than cmf_workspace_bytes()    */
    CMF_ECUDA = 3,         /* a CUDA runtime call failed                      */
    CMF_ETIMEOUT = 4,      /* a bounded device-side wait ran out              */
    CMF_NOT_CONVERGED = 5  /* status, not failure: max_iter reached first     */
} cmf_status;

typedef enum {
    CMF_PADMM = 0,      /* pADMMI: rpADMMI with r = 1                        */
    CMF_RPADMM_FG = 1,  /* rpADMMI, relaxation r on u (Fortin-Glowinski)     */
    CMF_RPADMM_EB = 2,  /* rpADMMII, relaxation rho (Eckstein-Bertsekas)     */
    CMF_RPDRQ = 3,      /* relaxed preconditioned Douglas-Rachford           */
    CMF_TY = 4,         /* pADMM-TY: the classical multi-block ADMM the paper
                           compares against (Eq. ADMM:Tai_yuan / Eq.
                           mADMM:Tai_yuan), sequential p-steps, no relaxation,
                           no convergence guarantee                           */
    CMF_CP = 5          /* ALG1: the first-order primal-dual (Chambolle-Pock)
                           method of the paper's Appendix (Eq. iteration:pd:seg
                           / Eq. alg1:4labels), step sizes sigma, tau with
                           sigma tau ||K*K|| < 1; fused and plain forms, the
                           state between calls is (u, q, p)                   */
} cmf_algo;

typedef enum { CMF_F32 = 0, CMF_F16 = 1, CMF_BF16 = 2 } cmf_dtype;

typedef enum {
    CMF_FUSED = 0,      /* one fused kernel per iteration (default)          */
    CMF_PLAIN = 1       /* one kernel per step of the method (baseline)      */
} cmf_impl;

/* Parameters.  cmf_default_params() fills the paper's values (Sec. 4):
 * c = 0.3, a = 8, a1 = 2 (binary a~), a2 = 2L, rho = 1.9, r = 1.618,
 * rPDRQ sigma = 0.2, tau = 1.0 (binary) or sigma = 5, tau = 0.4 (Potts),
 * ALG1 sigma = 0.4, tau = 1 / (10 sigma) (binary: ||K*K|| < 10) or
 * 1 / ((9 + L) sigma) (Potts, L > 2), one sRBGS sweep, isotropic P_alpha.
 * (L = 2 means the binary model; a two-label Potts ALG1 run needs
 * tau <= 1 / (11 sigma).) */
typedef struct {
    int algo;          /* cmf_algo                                             */
    int storage;       /* cmf_dtype of the flow planes                         */
    int impl;          /* cmf_impl                                             */
    int aniso;         /* 0: |q(x)|_2 <= alpha(x); 1: |q_k(x)| <= alpha(x)      */
    int sweeps;        /* symmetric red-black GS sweeps per rPDRQ step (>= 1)  */
    int max_iter;      /* cmf_solve_*: iteration cap                           */
    int check_every;   /* cmf_solve_*: iterations between certificate checks   */
    int warm_start;    /* cmf_solve_*: 0 = cold start, 1 = start from buffers  */
    int use_graph;     /* cmf_solve_*: 1 = device-driven loop (a CUDA graph whose
                          conditional WHILE node repeats {check_every iterations,
                          certificates, stop test} with no host round trip; used
                          when max_iter % check_every == 0), else a host-driven
                          loop; both give identical results                  */
    int variant;       /* kernel variant of the fused ADMM algorithms:
                          0 = automatic: warp strips where the layout allows
                          them (binary ADMM: two iterations per launch, as 4),
                          else TMA-staged tiles (Potts, and binary grids
                          of at most 2^21 pixels) where rows and planes are
                          16-byte aligned, else shared-memory tiles;
                          1 = shared-memory tiles;
                          2 = warp strips (even W and pitch, planes aligned to
                          two elements; for Potts the multipliers are kept as
                          u - cu p_s between the iterations of one call);
                          4 = binary ADMM: warp strips making two iterations
                          per launch (the intermediate state stays on chip;
                          an even number of such launches per call, single
                          ones for the rest and for scheduled rho_k; same
                          results as 2); Potts and rPDRQ: as 2;
                          8 / 16 / 32 = TMA tiles of that many rows         */
    double c;          /* ADMM step size                                       */
    double a;          /* q preconditioner N = a c I (a >= 8, Thm 1)           */
    double a1;         /* p preconditioner a~ (binary) / a_1 (Potts), >= 2     */
    double a2;         /* Potts p_s preconditioner a_2 >= 2L (Thm 2); 0 => 2L  */
    double rho;        /* rpADMMII / rPDRQ relaxation in (0, 2)                */
    double r;          /* rpADMMI relaxation in (0, (1+sqrt 5)/2)              */
    double sigma;      /* rPDRQ step sizes                                     */
    double tau;
    double tol_gap;    /* cmf_solve_*: stop when the relative gap <= tol_gap   */
    int costs;         /* Potts cost input: 0 = L float32 cost planes
                          [L][H][pitch] at d_C; 1 = computed where read (no
                          counterpart in the paper's statement, which takes the
                          costs as given): d_C holds one image plane I
                          [H][pitch] followed by the L levels c_i (floats), and
                          C_i(x) = (I(x) - c_i)^2; 2 = L float16 cost planes
                          [L][H][pitch] at d_C (the given costs rounded to
                          float16; every use converts them to float32).
                          Binary calls and batches need 0.                    */
    const double *rho_schedule; /* relaxation sequence {rho_k} of rpADMMII and
                          rPDRQ (Thm 1 and Thm 2 assume a non-decreasing
                          sequence in (0, 2); Sec. 4 takes rho_k = 1.9 for all
                          k).  Iteration k, counted from 0 at the first
                          iteration of a cmf_iterate_* or cmf_solve_* call
                          (warm starts included), uses rho_schedule[k] for
                          k < rho_schedule_len and rho from then on.  Host
                          array, read during the call only; NULL with length
                          0 (the default) means rho_k = rho.  CMF_EINVAL unless
                          every entry is in (0, 2), the entries do not
                          decrease, the last is <= rho and algo is rpADMMII or
                          rPDRQ; batches need length 0.  A solve runs the
                          scheduled iterations from the host, one launch per
                          iteration, and the rest as usual.              */
    int rho_schedule_len;
    int phase_storage; /* cmf_solve_potts only (no counterpart in the paper; a
                          storage schedule): 0 = off; CMF_F16 or CMF_BF16 = a
                          two-phase solve.  p->storage must be CMF_F32 (the
                          caller's buffers) and the solve starts cold.  Phase
                          one runs in phase_storage (flows q_i, p_i in 16 bits;
                          u, p_s float32) in state sets inside the workspace
                          until the certified gap is <= phase_gap, or is
                          below 10 phase_gap and above 0.7 times its value
                          at the check ceil(200 / check_every) checks
                          earlier (tested at every such check, from the
                          first on; the 16-bit rounding floor of
                          the instance: rounding of q_i and p_i holds the
                          16-label 4096^2 workload near 3e-4 in float16,
                          near 3e-3 in bfloat16, higher for larger c); the
                          state is then written exactly into the caller's
                          float32 buffers and phase two continues in float32
                          to tol_gap.  Iteration counts and history rows run
                          on across the switch; phase one alone may use up
                          max_iter.  phase_gap must lie above tol_gap.    */
    double phase_gap;
    int tune_step;     /* cmf_autotune_*: 0 = launch configurations only; 1 =
                          also the ADMM step size c of pADMMI, rpADMMI,
                          rpADMMII and pADMM-TY (candidates c, 2c, 4c, 8c
                          with the given kernel variant; Sec. 4 takes c = 0.3,
                          and any c > 0 keeps the convergence results of Thm 1
                          and Thm 2), and for a two-phase solve each of them
                          also with phase_gap = 1.5 tol_gap (the switch left
                          to the first phase's stall test).  Other algorithms
                          ignore it.                                         */
    int batch_rows;    /* cmf_solve_batch: band height of the warp-strip items
                          of its Potts instances, 8..24 (0 = 24); the items
                          of a band share its halo rows, the warps of a batch
                          share the work of small instances.               */
} cmf_params;

/* Fill *p with the paper's defaults for `algo` and L labels (L = 2 for the
 * binary model).  Returns CMF_EINVAL on a NULL pointer or unknown algo. */
cmf_status cmf_default_params(int algo, int L, cmf_params *p);

/* Human-readable name of a status code (static string). */
const char *cmf_status_str(cmf_status s);

/* Bytes of device workspace the calls below need for an H x W grid with L
 * labels (L = 2: binary) and row pitch `pitch`.  The workspace is caller-
 * owned device memory, at least 256-byte aligned, passed as d_ws/ws_bytes.
 * It holds one extra state set (two for the fused binary form; two 16-bit
 * sets more for a two-phase Potts solve), the plain form's temporaries, two
 * float32 planes of sum_i u_i for fused Potts rPDRQ, the certificate
 * partials, the solve loop's control block and max_iter / check_every + 1
 * history rows, so it depends on *p:
 * size it with the parameters the calls will use (a call whose parameters
 * need more returns CMF_ENOMEM before launching anything). */
size_t cmf_workspace_bytes(int H, int W, int L, int pitch, const cmf_params *p);
/* Device memory outside the workspace: the device-driven loop of cmf_solve_*
 * (use_graph = 1) keeps the instantiated CUDA graphs of the 8 most recently
 * used call signatures (see cmf_release_graphs).  Their memory is the
 * driver's (graph nodes and kernel parameters, a few KB to tens of KB per
 * graph); it is not part of cmf_workspace_bytes and is returned by
 * cmf_release_graphs. */

/* ------------------------------------------------------------------------ */
/* Binary model.  Planes: d_Cs, d_Ct (float32, read only); d_alpha (float32  */
/* plane or NULL, then alpha0 everywhere); state d_u (float32), d_qx, d_qy,  */
/* d_ps, d_pt (storage dtype).  For rPDRQ the flow buffers hold the          */
/* relaxed DR iterate (qbar, pbar_s, pbar_t) of Eq. iteration:quadratic:seg. */
/* ------------------------------------------------------------------------ */

/* Cold start: the alpha = 0 saddle point (u = 1 where C_t < C_s, q = 0,
 * p_s = p_t = min(C_s, C_t)); rPDRQ stores ybar = y - tau K u of that point. */
cmf_status cmf_init_binary(const float *d_Cs, const float *d_Ct, int H, int W, int pitch,
                           const cmf_params *p, float *d_u, void *d_qx, void *d_qy,
                           void *d_ps, void *d_pt, void *stream);

/* Exactly n_iter iterations of p->algo from the state in the buffers
 * (Eq. rpADMMI / Eq. rpADMMII / Eq. iteration:quadratic:seg); the result is
 * written back to the same buffers. */
cmf_status cmf_iterate_binary(const float *d_Cs, const float *d_Ct, const float *d_alpha,
                              float alpha0, int H, int W, int pitch, const cmf_params *p,
                              int n_iter, float *d_u, void *d_qx, void *d_qy, void *d_ps,
                              void *d_pt, void *d_ws, size_t ws_bytes, void *stream);

/* Certificates of the current state, into h_out[0..3] (host):
 *  E   = sum (1-ub) C_s + ub C_t + alpha |grad ub|, ub = clip(u, 0, 1)
 *  D   = sum min(C_s, C_t + div q)   (max-flow value of feasible q)
 *  gap = (E - D) / max(|E|, 1e-30)
 *  res = || div q - p_s + p_t ||_2
 * For rPDRQ the flows are y = ybar + tau K u and D uses P_alpha(q). */
cmf_status cmf_eval_binary(const float *d_Cs, const float *d_Ct, const float *d_alpha,
                           float alpha0, int H, int W, int pitch, const cmf_params *p,
                           const float *d_u, const void *d_qx, const void *d_qy,
                           const void *d_ps, const void *d_pt, double *h_out, void *d_ws,
                           size_t ws_bytes, void *stream);

/* Certificates of a binary state exactly as cmf_eval_binary computes them
 * (every algorithm, every storage type), for callers that cannot allocate
 * device memory when they need them (plug-ins that only receive a stream and
 * the solver's buffers from a host application that owns every allocation;
 * loops with a memory budget fixed up front).  It takes no workspace and
 * allocates nothing: its scratch is a static device array inside libcmf of
 * 393,248 bytes (per-block partial sums for up to 16384 blocks of 32 x 32
 * pixels, i.e. grids up to 4096 x 4096 pixels, plus the reduced scalars),
 * present on every GPU that loads the library until the process exits.
 *  - Larger grids (more than 16384 blocks of 32 x 32) return CMF_EINVAL.
 *  - Every call looks up the array's device address on the current device
 *    (cudaGetSymbolAddress), so calls after cudaDeviceReset stay valid.
 *  - The call cannot be captured into a CUDA graph: it synchronises `stream`
 *    and copies to the host.  On a stream that is being captured it returns
 *    CMF_EINVAL before launching anything, and the capture stays valid.
 *  - All calls share the array: calls whose GPU work overlaps (different
 *    streams, or different host threads on one device) race and give wrong
 *    results.  Nothing in the array has to start at zero; each call
 *    overwrites what it reads.
 *  - Like cmf_eval_binary it synchronises `stream` and writes h_out[0..3]
 *    = (E, D, gap, res) on the host.
 * The paper has no counterpart: this is a deployment variant of
 * cmf_eval_binary. */
cmf_status cmf_eval_binary_noalloc(const float *d_Cs, const float *d_Ct, const float *d_alpha,
                                   float alpha0, int H, int W, int pitch, const cmf_params *p,
                                   const float *d_u, const void *d_qx, const void *d_qy,
                                   const void *d_ps, const void *d_pt, double *h_out,
                                   void *stream);

/* Solve to gap <= p->tol_gap or p->max_iter iterations: cold start unless
 * p->warm_start, then repeat {check_every iterations; certificates}.
 * h_hist (host, may be NULL) receives up to hist_cap rows of
 * (iteration, E, D, gap, res); *h_iters (host, may be NULL) the iterations
 * run.  Returns CMF_OK on convergence, CMF_NOT_CONVERGED at max_iter. */
cmf_status cmf_solve_binary(const float *d_Cs, const float *d_Ct, const float *d_alpha,
                            float alpha0, int H, int W, int pitch, const cmf_params *p,
                            float *d_u, void *d_qx, void *d_qy, void *d_ps, void *d_pt,
                            double *h_hist, int hist_cap, int *h_iters, void *d_ws,
                            size_t ws_bytes, void *stream);

/* The device-driven loop of cmf_solve_* (use_graph = 1) is a CUDA graph
 * whose kernels have the call's pointers, sizes and coefficients baked in.
 * It is built and instantiated on the first call with a given signature --
 * the current device, the model, L, H, W, pitch, alpha0, every device
 * pointer (costs, alpha, state, workspace) and *p apart from warm_start and
 * the rho schedule -- and replayed by later calls with the same signature
 * (a solve called in a loop pays the graph construction once).  The
 * executable graphs of the 8 most recently used signatures are kept, in
 * device memory the library allocates.  A replay only needs buffers of the
 * signature's sizes at the signature's addresses, whatever they hold, so
 * freeing and reallocating buffers never makes a kept graph wrong; a graph
 * whose buffers are gone is simply never matched again.
 * cmf_release_graphs() destroys them all, to return their memory.
 * Thread-safe; graphs still running are freed when they complete.  No
 * counterpart in the paper. */
cmf_status cmf_release_graphs(void);

/* ------------------------------------------------------------------------ */
/* Potts model, L labels (2 <= L <= 64).  d_C: L cost planes C_1..C_L      */
/* (float32, or see cmf_params.costs).  State: d_u (L float32 planes),      */
/* d_qx, d_qy, d_p (L planes each, storage dtype), d_ps (one float32        */
/* plane).  rPDRQ: (qbar_i, pbar_i, pbar_s).                                */
/* ------------------------------------------------------------------------ */

/* Cold start: u_i = 1 for the first cheapest label, q_i = 0,
 * p_i = p_s = min_j C_j; rPDRQ stores ybar = y - tau K u of that point. */
cmf_status cmf_init_potts(const float *d_C, int L, int H, int W, int pitch,
                          const cmf_params *p, float *d_u, void *d_qx, void *d_qy, void *d_p,
                          void *d_ps, void *stream);

/* Exactly n_iter iterations (Eq. multi:fg:4, the Eckstein-Bertsekas Potts
 * equations after Thm 2, Eq. pdrq:4labels), in place. */
cmf_status cmf_iterate_potts(const float *d_C, int L, const float *d_alpha, float alpha0, int H,
                             int W, int pitch, const cmf_params *p, int n_iter, float *d_u,
                             void *d_qx, void *d_qy, void *d_p, void *d_ps, void *d_ws,
                             size_t ws_bytes, void *stream);

/* Certificates into h_out[0..3]:
 *  E   = sum_i sum_x ub_i C_i + alpha |grad ub_i|, ub(x) = simplex projection
 *  D   = sum_x min_i (C_i + div q_i)
 *  gap = (E - D) / max(|E|, 1e-30),  res = || div q_i - p_s + p_i ||_2. */
cmf_status cmf_eval_potts(const float *d_C, int L, const float *d_alpha, float alpha0, int H,
                          int W, int pitch, const cmf_params *p, const float *d_u,
                          const void *d_qx, const void *d_qy, const void *d_p, const void *d_ps,
                          double *h_out, void *d_ws, size_t ws_bytes, void *stream);

/* Solve the Potts model (Eq. potts-mf, dual of Eq. relaxed-potts) to a
 * relative gap <= p->tol_gap or p->max_iter iterations, as cmf_solve_binary
 * does for the binary model: cold start (u_i = 1 for the first cheapest
 * label, q_i = 0, p_i = p_s = min_j C_j) unless p->warm_start, then repeat
 * {check_every iterations of p->algo (Eq. multi:fg:4, the Eckstein-Bertsekas
 * equations after Thm 2, Eq. pdrq:4labels, Eq. mADMM:Tai_yuan, Eq.
 * alg1:4labels); the certificates of cmf_eval_potts}.  h_hist (host, may be
 * NULL) receives up to hist_cap rows of (iteration, E, D, gap, res); *h_iters
 * (host, may be NULL) the iterations run.  The state buffers hold the last
 * iterate (u itself, also for the warp-strip kernels' w form).  Returns
 * CMF_OK on convergence, CMF_NOT_CONVERGED at max_iter, CMF_ETIMEOUT when a
 * bounded device wait ran out. */
cmf_status cmf_solve_potts(const float *d_C, int L, const float *d_alpha, float alpha0, int H,
                           int W, int pitch, const cmf_params *p, float *d_u, void *d_qx,
                           void *d_qy, void *d_p, void *d_ps, double *h_hist, int hist_cap,
                           int *h_iters, void *d_ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Autotuning (no counterpart in the paper: a launch-configuration search).  */
/* Solves the problem from a cold start once per candidate configuration --  */
/* the kernel variant (1, 2, 4 (binary), 8, 16, 32) of the fused ADMM       */
/* algorithms, or the sRBGS sweep count (1, 2, 3) of fused rPDRQ, and with   */
/* p->tune_step = 1 the ADMM step size c (c, 2c, 4c, 8c) -- with everything  */
/* else taken from *p, and writes the candidate with the shortest time to   */
/* p->tol_gap                                                               */
/* (CUDA events on `stream`, best of two runs after a warm-up) to *best and  */
/* its time in milliseconds to *h_best_ms (host, may be NULL).  The state    */
/* buffers are overwritten (they hold the last trial's solution).  Returns  */
/* CMF_NOT_CONVERGED when no candidate reached the gap within max_iter.     */
/* ------------------------------------------------------------------------ */
cmf_status cmf_autotune_binary(const float *d_Cs, const float *d_Ct, const float *d_alpha,
                               float alpha0, int H, int W, int pitch, const cmf_params *p,
                               float *d_u, void *d_qx, void *d_qy, void *d_ps, void *d_pt,
                               void *d_ws, size_t ws_bytes, cmf_params *best,
                               double *h_best_ms, void *stream);

cmf_status cmf_autotune_potts(const float *d_C, int L, const float *d_alpha, float alpha0,
                              int H, int W, int pitch, const cmf_params *p, float *d_u,
                              void *d_qx, void *d_qy, void *d_p, void *d_ps, void *d_ws,
                              size_t ws_bytes, cmf_params *best, double *h_best_ms,
                              void *stream);

/* ------------------------------------------------------------------------ */
/* Batches: many binary and Potts instances of uneven size and label count  */
/* solved together in one device-driven loop (a CUDA graph whose            */
/* conditional WHILE node repeats {check_every iterations of every active   */
/* instance, certificates, per-instance stop test}).  Converged instances   */
/* stop iterating (per-instance convergence masks); the loop ends when all  */
/* have converged or reached max_iter.  p->use_graph = 0 runs the same      */
/* chunks host-driven (the stop flag read back after each), with the same   */
/* results: for profilers and drivers without conditional graph nodes.      */
/* ------------------------------------------------------------------------ */

typedef struct {
    /* problem (inputs) */
    int model;              /* 0 = binary (L must be 2), 1 = Potts              */
    int L, H, W, pitch;     /* labels, grid, row stride in elements             */
    const float *d_cost;    /* binary: C_s then C_t (2 planes); Potts: L planes */
    const float *d_alpha;   /* alpha plane or NULL (then alpha0)                */
    float alpha0;
    /* state (in/out, caller-owned device buffers, as in the single solvers)   */
    float *d_u;             /* binary: 1 plane; Potts: L planes (float32)       */
    void *d_qx, *d_qy;      /* 1 / L planes each, storage dtype                 */
    void *d_p;              /* binary: p_t (1 plane); Potts: p_i (L planes)     */
    void *d_ps;             /* p_s (1 plane; Potts: float32)                    */
    /* results (outputs) */
    int iters;              /* iterations run for this instance                 */
    int status;             /* CMF_OK or CMF_NOT_CONVERGED                      */
    double energy, dual, gap, res;  /* last certificates (as cmf_eval_*)       */
} cmf_instance;

/* Workspace bytes for a batch (0 when an instance or the parameters are
 * invalid).  The batch runs the fused kernels (p->impl = CMF_FUSED), needs an
 * even p->check_every that divides p->max_iter, and for rPDRQ one sweep. */
size_t cmf_batch_workspace_bytes(const cmf_instance *inst, int n, const cmf_params *p);

/* Solve all n instances (host array; device pointers inside) with the same
 * algorithm and parameters (rPDRQ: the same sigma and tau for every
 * instance; Potts instances use a2 = max(p->a2, 2L), the bound of Thm 2;
 * ALG1 instances use tau = min(p->tau, 1 / ((L == 2 ? 10 : 9 + L) sigma)),
 * the step bound cmf_default_params takes for their L);
 * cold start unless p->warm_start.  Fills the
 * result fields of every instance.  Returns CMF_OK when every instance
 * reached p->tol_gap, CMF_NOT_CONVERGED when some stopped at max_iter. */
cmf_status cmf_solve_batch(cmf_instance *inst, int n, const cmf_params *p, void *d_ws,
                           size_t ws_bytes, void *stream);

/* Time cmf_solve_batch (cold starts; the instances' state buffers are
 * overwritten) over candidate launch and check settings and write the
 * fastest whose every instance reaches p->tol_gap to *best: check_every in
 * {k, 2k, 5k} (k = p->check_every; those that divide p->max_iter) and,
 * when the batch has strip instances, batch_rows in {12, 16, 24}.  The
 * workspace must hold cmf_batch_workspace_bytes for batch_rows = 12 (the
 * largest item tables).  *h_best_ms: the fastest time.  Returns
 * CMF_NOT_CONVERGED when no candidate converged. */
cmf_status cmf_autotune_batch(cmf_instance *inst, int n, const cmf_params *p, cmf_params *best,
                              double *h_best_ms, void *d_ws, size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CMF_H */
