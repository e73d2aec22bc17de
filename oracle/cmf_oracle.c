/*
 * cmf_oracle.c -- plain, slow FP64 CPU oracle for continuous max-flow /
 * min-cut (Sun, Tai, Yuan, "Efficient ADMM and splitting methods for
 * continuous min-cut and max-flow problems").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: it exists so the tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA solver against an
 * independent transcription of the paper.  It shares no code, header or
 * constant with the CUDA library.
 *
 * Everything is double precision, full-grid loops, one array per quantity,
 * one step of the paper per loop, in the paper's order.  Arrays are dense
 * row-major H x W (index i*W + j; i = row = e2 direction, j = column = e1
 * direction).  Potts planes are stacked [L][H][W].
 *
 * Readings where the paper is silent or garbled (each is tested):
 *  - Discretisation (Sec. 3.1, Thm 1 cites the standard scheme with
 *    ||div* div|| <= 8): unit spacing, forward-difference gradient that is 0
 *    on the far boundary, div = -grad^T.
 *  - Conservation sign: div q - p_s + p_t = 0 (binary) and
 *    div q_i - p_s + p_i = 0 (Potts), as in the augmented Lagrangians
 *    (Eq. augfunc:twolabel, Eq. multi:aug:func) and every update formula.
 *  - P_alpha with alpha(x) = 0 returns 0 (Eq. projections divides by alpha).
 *  - Potts rpADMMII multiplier step: no rho on (p_i^{k+1} - p_s^{k+1}),
 *    following the general Eckstein-Bertsekas update (Eq.
 *    update:two:sun:lag) and the binary rpADMMII; the printed Potts variant
 *    is available through `literal_potts_u`.
 *  - Binary rPDRQ p_s reflection: prox of -tau<1,p_s> adds +tau, as in the
 *    Potts rPDRQ (Eq. pdrq:4labels).
 *  - Potts a2 = 2L (Eq. multilabel:pre:p); rPDRQ for general L uses
 *    (L-1) in b_i and T_0 = -Lap + (L+1) I (Lemma 1).
 *  - ALG1 (Chambolle-Pock, Appendix): the binary p_s step adds +sigma (prox
 *    of -sigma<1,p_s>, as in its Potts form); the Potts q_i step uses the
 *    extrapolated ubar_i of the general scheme (Eq. alg:pd), not u_i.  The
 *    state between calls is (u, q, p); a run recovers ubar^k = 2u^k - u^{k-1}
 *    from u^k - u^{k-1} = -tau (div q + p_t - p_s)^k, which its own
 *    multiplier step makes exact.
 *  - Cold start (the paper gives none): the alpha = 0 saddle point, i.e.
 *    q = 0, p = min cost, u = indicator of the cheapest label; rPDRQ holds
 *    ybar = y - tau K u of that point.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_PADMM = 0, ORC_RPADMM_FG = 1, ORC_RPADMM_EB = 2, ORC_RPDRQ = 3, ORC_TY = 4,
       ORC_CP = 5 };

/* Parameters of one run.  Mirrored by a ctypes.Structure in __init__.py. */
typedef struct {
    int algo;          /* ORC_* above                                     */
    int aniso;         /* 0: |q(x)|_2 <= alpha(x); 1: |q_k(x)| <= alpha(x)  */
    int sweeps;        /* symmetric red-black GS sweeps per rPDRQ step      */
    int literal_potts_u; /* 1: printed Potts rpADMMII u-step (extra rho)    */
    double c;          /* ADMM step size (0.3 in Sec. 4)                   */
    double a;          /* q preconditioner N = a c I, a >= ||div* div||     */
    double a1;         /* p preconditioner (binary: a~; Potts: a_1)         */
    double a2;         /* Potts p_s preconditioner a_2 (>= 2L)              */
    double rho;        /* EB / DR relaxation                                */
    double r;          /* FG relaxation on u                               */
    double sigma, tau; /* rPDRQ and ALG1 step sizes                         */
} orc_params;

#define AT(a, i, j) ((a)[(size_t)(i) * (size_t)W + (size_t)(j)])

/* Element-wise loops (each iteration writes only its own elements) may run on
 * several threads when the oracle is built with OpenMP; results are the same
 * for any thread count.  Sums stay sequential. */
#ifdef _OPENMP
#define ORC_PRAGMA(x) _Pragma(#x)
#define ORC_PAR_FOR(n) ORC_PRAGMA(omp parallel for schedule(static) if ((n) > 32768))
#else
#define ORC_PAR_FOR(n)
#endif

static double *dalloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

#ifdef _OPENMP
#include <omp.h>
#endif
/* Threads for the element-wise loops (n < 1: leave the setting alone);
 * returns the number that will be used (1 without OpenMP). */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Discrete operators                                                        */
/* ------------------------------------------------------------------------ */

/* grad g = (g(i,j+1)-g(i,j), g(i+1,j)-g(i,j)); 0 where the neighbour is
 * outside the grid. */
void orc_grad(int H, int W, const double *g, double *gx, double *gy) {
    ORC_PAR_FOR((size_t)H * W)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            AT(gx, i, j) = (j < W - 1) ? AT(g, i, j + 1) - AT(g, i, j) : 0.0;
            AT(gy, i, j) = (i < H - 1) ? AT(g, i + 1, j) - AT(g, i, j) : 0.0;
        }
}

/* div q = -grad^T q.  Entry (i,j) collects +q(i,j) from the forward
 * difference that starts at (i,j) and -q(i,j-1) / -q(i-1,j) from the ones
 * that end there; components that grad never produces (the far-boundary
 * ones) do not contribute. */
void orc_div(int H, int W, const double *qx, const double *qy, double *d) {
    ORC_PAR_FOR((size_t)H * W)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double v = 0.0;
            if (j < W - 1) v += AT(qx, i, j);
            if (j > 0) v -= AT(qx, i, j - 1);
            if (i < H - 1) v += AT(qy, i, j);
            if (i > 0) v -= AT(qy, i - 1, j);
            AT(d, i, j) = v;
        }
}

/* div^* = -grad (the adjoint of div), written as its own step so the q-update
 * reads like (I - (1/a) div^* div) q in the paper. */
static void orc_div_adjoint(int H, int W, const double *w, double *ox, double *oy) {
    orc_grad(H, W, w, ox, oy);
    ORC_PAR_FOR((size_t)H * W)
    for (size_t k = 0; k < (size_t)H * W; ++k) { ox[k] = -ox[k]; oy[k] = -oy[k]; }
}

/* P_alpha (Eq. projections): q / max(1, |q|/alpha); alpha = 0 gives 0.
 * Anisotropic option: clamp each component to [-alpha, alpha]. */
void orc_project_alpha(size_t n, double *qx, double *qy, const double *alpha, int aniso) {
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        double al = alpha[k];
        if (aniso) {
            if (qx[k] > al) qx[k] = al;
            if (qx[k] < -al) qx[k] = -al;
            if (qy[k] > al) qy[k] = al;
            if (qy[k] < -al) qy[k] = -al;
            continue;
        }
        if (al <= 0.0) { qx[k] = 0.0; qy[k] = 0.0; continue; }
        double nrm = sqrt(qx[k] * qx[k] + qy[k] * qy[k]);
        double den = nrm / al > 1.0 ? nrm / al : 1.0;
        qx[k] /= den;
        qy[k] /= den;
    }
}

static double dmin(double x, double y) { return x < y ? x : y; }

/* One symmetric red-black Gauss-Seidel sweep, repeated `sweeps` times, for
 * T u = b with T = st (kappa I - Lap) and the 5-point Neumann Laplacian:
 * T_xx = st (kappa + n_nb(x)), T_x,nb = -st.  Red = (i+j) even.  A symmetric
 * sweep is red, black, black, red; the second black pass reproduces the first
 * (its red neighbours have not changed), so one sweep is red, black, red and
 * s sweeps are red, (black, red) x s.  One sweep from u equals
 * u + M^{-1} (b - T u) with M the sRBGS preconditioner of T (Eq.
 * iteration:quadratic:seg, Eq. pdrq:4labels). */
static void orc_halfsweep(int H, int W, double kappa, double st, const double *b, double *u,
                          int colour) {
    ORC_PAR_FOR((size_t)H * W)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            if (((i + j) & 1) != colour) continue;
            double rhs = AT(b, i, j);
            int nnb = 0;
            if (j > 0) { rhs += st * AT(u, i, j - 1); ++nnb; }
            if (j < W - 1) { rhs += st * AT(u, i, j + 1); ++nnb; }
            if (i > 0) { rhs += st * AT(u, i - 1, j); ++nnb; }
            if (i < H - 1) { rhs += st * AT(u, i + 1, j); ++nnb; }
            AT(u, i, j) = rhs / (st * (kappa + nnb));
        }
}

void orc_srbgs(int H, int W, double kappa, double st, const double *b, double *u, int sweeps) {
    orc_halfsweep(H, W, kappa, st, b, u, 0);
    for (int s = 0; s < sweeps; ++s) {
        orc_halfsweep(H, W, kappa, st, b, u, 1);
        orc_halfsweep(H, W, kappa, st, b, u, 0);
    }
}

/* Euclidean projection of v (length n) onto the unit simplex, by sorting
 * (Held, Wolfe & Crowder 1974; Duchi et al. 2008). */
static int cmp_desc(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}
int orc_simplex(int n, const double *v, double *w) {
    if (n < 1 || n > 64) return -1; /* the sort buffer holds 64 entries */
    double s[64];
    memcpy(s, v, (size_t)n * sizeof(double));
    qsort(s, (size_t)n, sizeof(double), cmp_desc);
    double cum = 0.0, theta = 0.0;
    for (int k = 0; k < n; ++k) {
        cum += s[k];
        double t = (cum - 1.0) / (k + 1);
        if (s[k] - t > 0.0) theta = t;
    }
    for (int k = 0; k < n; ++k) w[k] = v[k] - theta > 0.0 ? v[k] - theta : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Binary model: Eq. two-label-mf                                            */
/* ------------------------------------------------------------------------ */

/* Cold start: the alpha = 0 saddle point. u = 1 where C_t < C_s (u = 1
 * costs C_t), q = 0, p_s = p_t = min(C_s, C_t).  rPDRQ keeps ybar instead of
 * y; at a fixed point y = ybar + tau K u (Eq. iteration:quadratic:seg), so it
 * starts from ybar = y - tau K u: qbar = tau grad u, pbar_t = p_t - tau u,
 * pbar_s = p_s + tau u.  This start is a fixed point when alpha = 0. */
void orc_binary_init(int H, int W, const double *Cs, const double *Ct, int dr, double tau,
                     double *u, double *qx, double *qy, double *ps, double *pt) {
    ORC_PAR_FOR((size_t)H * W)
    for (size_t k = 0; k < (size_t)H * W; ++k) {
        u[k] = Ct[k] < Cs[k] ? 1.0 : 0.0;
        qx[k] = 0.0;
        qy[k] = 0.0;
        ps[k] = pt[k] = dmin(Cs[k], Ct[k]);
    }
    if (!dr) return;
    orc_grad(H, W, u, qx, qy);
    ORC_PAR_FOR((size_t)H * W)
    for (size_t k = 0; k < (size_t)H * W; ++k) {
        qx[k] *= tau;
        qy[k] *= tau;
        pt[k] -= tau * u[k];
        ps[k] += tau * u[k];
    }
}

/* One rpADMMII (Eckstein-Bertsekas) or rpADMMI / pADMMI (Fortin-Glowinski)
 * iteration, Eq. rpADMMII / Eq. rpADMMI. */
static void binary_admm_step(int H, int W, const double *Cs, const double *Ct, const double *alpha,
                             const orc_params *P, double *u, double *qx, double *qy, double *ps,
                             double *pt, double *w1, double *w2, double *w3, double *w4,
                             double *w5) {
    const size_t n = (size_t)H * W;
    const double c = P->c, a = P->a, at = P->a1;
    const int eb = (P->algo == ORC_RPADMM_EB);
    const double rho = eb ? P->rho : 1.0;
    const double r = (P->algo == ORC_RPADMM_FG) ? P->r : 1.0;

    /* q^{k+1} = P_alpha((I - (1/a) div^* div) q^k + (1/a) grad(p_t - p_s - u/c)) */
    double *dq = w1, *sx = w2, *sy = w3, *gx = w4, *gy = w5;
    orc_div(H, W, qx, qy, dq);
    orc_div_adjoint(H, W, dq, sx, sy);
    double *h = dq; /* reuse: h = p_t - p_s - u/c */
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) h[k] = pt[k] - ps[k] - u[k] / c;
    orc_grad(H, W, h, gx, gy);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        qx[k] = qx[k] - sx[k] / a + gx[k] / a;
        qy[k] = qy[k] - sy[k] / a + gy[k] / a;
    }
    orc_project_alpha(n, qx, qy, alpha, P->aniso);

    /* p^{k+1}: both p_t and p_s read p^k (Jacobi). */
    double *d = w1;
    orc_div(H, W, qx, qy, d);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        double pt0 = pt[k], ps0 = ps[k];
        double pt1 = dmin(pt0 - (rho / at) * (pt0 - ps0) + (1.0 / at) * (-rho * d[k] + u[k] / c),
                          Ct[k]);
        double ps1 = dmin(ps0 - (rho / at) * (ps0 - pt0) +
                              (1.0 / at) * (rho * d[k] - u[k] / c + 1.0 / c),
                          Cs[k]);
        /* u^{k+1} */
        if (eb)
            u[k] = u[k] - c * ((pt1 - ps1) - (1.0 - rho) * (pt0 - ps0) + rho * d[k]);
        else
            u[k] = u[k] - r * c * ((pt1 - ps1) + d[k]);
        pt[k] = pt1;
        ps[k] = ps1;
    }
}

/* One rPDRQ iteration, Eq. iteration:quadratic:seg.  State (u, qbar, pbar_s,
 * pbar_t); K = (-grad; I; -I), K^* y = div q + p_t - p_s. */
static void binary_dr_step(int H, int W, const double *Cs, const double *Ct, const double *alpha,
                           const orc_params *P, double *u, double *qbx, double *qby, double *pbs,
                           double *pbt, double *w1, double *w2, double *w3, double *w4,
                           double *w5) {
    const size_t n = (size_t)H * W;
    const double sg = P->sigma, tau = P->tau, rho = P->rho;
    double *b = w1;
    orc_div(H, W, qbx, qby, b);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) b[k] = -sg * (b[k] + pbt[k] - pbs[k]);
    /* u^{k+1} = u^k + M^{-1}[b - T u^k], T = sigma tau (-Lap + 2I) */
    orc_srbgs(H, W, 2.0, sg * tau, b, u, P->sweeps);
    double *gx = w2, *gy = w3, *tx = w4, *ty = w5;
    orc_grad(H, W, u, gx, gy);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        double q1 = qbx[k] - tau * gx[k];
        double q2 = qby[k] - tau * gy[k];
        tx[k] = 2.0 * q1 - qbx[k];
        ty[k] = 2.0 * q2 - qby[k];
        gx[k] = q1; /* keep q^{k+1} */
        gy[k] = q2;
    }
    orc_project_alpha(n, tx, ty, alpha, P->aniso);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        double pt1 = pbt[k] + tau * u[k];
        double ps1 = pbs[k] - tau * u[k];
        qbx[k] = qbx[k] + rho * (tx[k] - gx[k]);
        qby[k] = qby[k] + rho * (ty[k] - gy[k]);
        pbt[k] = pbt[k] + rho * (dmin(2.0 * pt1 - pbt[k], Ct[k]) - pt1);
        pbs[k] = pbs[k] + rho * (dmin(2.0 * ps1 - pbs[k] + tau, Cs[k]) - ps1);
    }
}

/* One pADMM-TY iteration (Eq. ADMM:Tai_yuan): the q-step of the other ADMM
 * variants, then the sequential (Gauss-Seidel) maximisations of the
 * augmented Lagrangian over p_s (with p_t^k) and over p_t (with p_s^{k+1}),
 * then the multiplier step u^{k+1} = u^k - c (p_t - p_s + div q)^{k+1}. */
static void binary_ty_step(int H, int W, const double *Cs, const double *Ct, const double *alpha,
                           const orc_params *P, double *u, double *qx, double *qy, double *ps,
                           double *pt, double *w1, double *w2, double *w3, double *w4,
                           double *w5) {
    const size_t n = (size_t)H * W;
    const double c = P->c, a = P->a;
    double *dq = w1, *sx = w2, *sy = w3, *gx = w4, *gy = w5;
    orc_div(H, W, qx, qy, dq);
    orc_div_adjoint(H, W, dq, sx, sy);
    double *h = dq;
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) h[k] = pt[k] - ps[k] - u[k] / c;
    orc_grad(H, W, h, gx, gy);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        qx[k] = qx[k] - sx[k] / a + gx[k] / a;
        qy[k] = qy[k] - sy[k] / a + gy[k] / a;
    }
    orc_project_alpha(n, qx, qy, alpha, P->aniso);
    double *d = w1;
    orc_div(H, W, qx, qy, d);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        ps[k] = dmin(pt[k] + d[k] - u[k] / c + 1.0 / c, Cs[k]);
        pt[k] = dmin(ps[k] - d[k] + u[k] / c, Ct[k]);
        u[k] = u[k] - c * (pt[k] - ps[k] + d[k]);
    }
}

/* ubar = u - tau (div q + p_t - p_s): the extrapolated multiplier of ALG1
 * recovered from the state (see the readings above). */
static void binary_cp_ubar(int H, int W, double tau, const double *u, const double *qx,
                           const double *qy, const double *ps, const double *pt, double *ubar) {
    const size_t n = (size_t)H * W;
    orc_div(H, W, qx, qy, ubar);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) ubar[k] = u[k] - tau * (ubar[k] + pt[k] - ps[k]);
}

/* One ALG1 iteration (Chambolle-Pock, Eq. iteration:pd:seg): dual steps on
 * q, p_t, p_s with the extrapolated ubar^k, the primal step on u, then
 * ubar^{k+1} = 2 u^{k+1} - u^k. */
static void binary_cp_step(int H, int W, const double *Cs, const double *Ct, const double *alpha,
                           const orc_params *P, double *u, double *qx, double *qy, double *ps,
                           double *pt, double *ubar, double *w1, double *w2, double *w3) {
    const size_t n = (size_t)H * W;
    const double sg = P->sigma, tau = P->tau;
    double *gx = w1, *gy = w2, *d = w3;
    orc_grad(H, W, ubar, gx, gy);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        qx[k] = qx[k] - sg * gx[k];
        qy[k] = qy[k] - sg * gy[k];
    }
    orc_project_alpha(n, qx, qy, alpha, P->aniso);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        pt[k] = dmin(pt[k] + sg * ubar[k], Ct[k]);
        ps[k] = dmin(ps[k] - sg * ubar[k] + sg, Cs[k]);
    }
    orc_div(H, W, qx, qy, d);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        const double u0 = u[k];
        u[k] = u0 - tau * (d[k] + pt[k] - ps[k]);
        ubar[k] = 2.0 * u[k] - u0;
    }
}

/* Run n_iter iterations from the given state (cold start first if
 * `cold` != 0).  Returns 0, or -1 on a bad algorithm code / allocation. */
int orc_binary_run(int H, int W, const double *Cs, const double *Ct, const double *alpha,
                   const orc_params *P, int n_iter, int cold, double *u, double *qx, double *qy,
                   double *ps, double *pt) {
    if (P->algo < ORC_PADMM || P->algo > ORC_CP) return -1;
    const size_t n = (size_t)H * W;
    if (cold) orc_binary_init(H, W, Cs, Ct, P->algo == ORC_RPDRQ, P->tau, u, qx, qy, ps, pt);
    double *w1 = dalloc(n), *w2 = dalloc(n), *w3 = dalloc(n), *w4 = dalloc(n), *w5 = dalloc(n);
    if (!w1 || !w2 || !w3 || !w4 || !w5) return -1;
    if (P->algo == ORC_CP) binary_cp_ubar(H, W, P->tau, u, qx, qy, ps, pt, w5);
    for (int it = 0; it < n_iter; ++it) {
        if (P->algo == ORC_CP)
            binary_cp_step(H, W, Cs, Ct, alpha, P, u, qx, qy, ps, pt, w5, w1, w2, w3);
        else if (P->algo == ORC_RPDRQ)
            binary_dr_step(H, W, Cs, Ct, alpha, P, u, qx, qy, ps, pt, w1, w2, w3, w4, w5);
        else if (P->algo == ORC_TY)
            binary_ty_step(H, W, Cs, Ct, alpha, P, u, qx, qy, ps, pt, w1, w2, w3, w4, w5);
        else
            binary_admm_step(H, W, Cs, Ct, alpha, P, u, qx, qy, ps, pt, w1, w2, w3, w4, w5);
    }
    free(w1); free(w2); free(w3); free(w4); free(w5);
    return 0;
}

/* Certificates of the binary state (out[0..3] = E, D, relative gap, l2
 * conservation residual).
 *  E(u) = sum (1-ub) C_s + ub C_t + alpha |grad ub|, ub = clip(u, 0, 1)
 *         (Eq. seg:chanvese; |.| Euclidean, or l1 when aniso).
 *  D(q) = sum min(C_s, C_t + div q), the max-flow value of the best p_s, p_t
 *         for a feasible q under div q - p_s + p_t = 0 (Eq. two-label-mf).
 *  gap  = (E - D) / max(|E|, 1e-30).
 *  res  = || div q - p_s + p_t ||_2.
 * For rPDRQ (dr != 0) the flows are y = ybar + tau K u and the dual is
 * evaluated at P_alpha(q), which is feasible and equals q at a fixed point. */
void orc_binary_eval(int H, int W, const double *Cs, const double *Ct, const double *alpha,
                     int aniso, int dr, double tau, const double *u, const double *qx,
                     const double *qy, const double *ps, const double *pt, double *out) {
    const size_t n = (size_t)H * W;
    double *ub = dalloc(n), *gx = dalloc(n), *gy = dalloc(n), *fx = dalloc(n), *fy = dalloc(n),
           *fs = dalloc(n), *ft = dalloc(n), *d = dalloc(n);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) ub[k] = u[k] < 0.0 ? 0.0 : (u[k] > 1.0 ? 1.0 : u[k]);
    orc_grad(H, W, ub, gx, gy);
    double E = 0.0;
    for (size_t k = 0; k < n; ++k) {
        double tv = aniso ? fabs(gx[k]) + fabs(gy[k]) : sqrt(gx[k] * gx[k] + gy[k] * gy[k]);
        E += (1.0 - ub[k]) * Cs[k] + ub[k] * Ct[k] + alpha[k] * tv;
    }
    if (dr) {
        orc_grad(H, W, u, gx, gy);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            fx[k] = qx[k] - tau * gx[k];
            fy[k] = qy[k] - tau * gy[k];
            ft[k] = pt[k] + tau * u[k];
            fs[k] = ps[k] - tau * u[k];
        }
    } else {
        memcpy(fx, qx, n * sizeof(double));
        memcpy(fy, qy, n * sizeof(double));
        memcpy(ft, pt, n * sizeof(double));
        memcpy(fs, ps, n * sizeof(double));
    }
    orc_div(H, W, fx, fy, d);
    double res = 0.0;
    for (size_t k = 0; k < n; ++k) {
        double rr = d[k] - fs[k] + ft[k];
        res += rr * rr;
    }
    orc_project_alpha(n, fx, fy, alpha, aniso);
    orc_div(H, W, fx, fy, d);
    double D = 0.0;
    for (size_t k = 0; k < n; ++k) D += dmin(Cs[k], Ct[k] + d[k]);
    out[0] = E;
    out[1] = D;
    out[2] = (E - D) / (fabs(E) > 1e-30 ? fabs(E) : 1e-30);
    out[3] = sqrt(res);
    free(ub); free(gx); free(gy); free(fx); free(fy); free(fs); free(ft); free(d);
}

/* ------------------------------------------------------------------------ */
/* Potts model: Eq. potts-mf, L labels                                       */
/* ------------------------------------------------------------------------ */

/* Cold start: the alpha = 0 saddle point. u_i = 1 for the first cheapest
 * label, q_i = 0, p_s = p_i = min_j C_j.  rPDRQ starts from ybar = y - tau K u:
 * qbar_i = tau grad u_i, pbar_i = p_i - tau u_i, pbar_s = p_s + tau sum_i u_i. */
void orc_potts_init(int H, int W, int L, const double *C, int dr, double tau, double *u,
                    double *qx, double *qy, double *p, double *ps) {
    const size_t n = (size_t)H * W;
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        int best = 0;
        for (int i = 1; i < L; ++i)
            if (C[i * n + k] < C[best * n + k]) best = i;
        double m = C[best * n + k];
        ps[k] = m;
        for (int i = 0; i < L; ++i) {
            u[i * n + k] = (i == best) ? 1.0 : 0.0;
            qx[i * n + k] = 0.0;
            qy[i * n + k] = 0.0;
            p[i * n + k] = m;
        }
    }
    if (!dr) return;
    for (int i = 0; i < L; ++i) {
        orc_grad(H, W, u + i * n, qx + i * n, qy + i * n);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            qx[i * n + k] *= tau;
            qy[i * n + k] *= tau;
            p[i * n + k] -= tau * u[i * n + k];
        }
    }
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) ps[k] += tau; /* sum_i u_i = 1 */
}

/* One Potts rpADMMII / rpADMMI / pADMMI iteration (Eqs. subequations after
 * Thm 2, Eq. multi:fg:4), for general L with a2 from the parameters. */
static void potts_admm_step(int H, int W, int L, const double *C, const double *alpha,
                            const orc_params *P, double *u, double *qx, double *qy, double *p,
                            double *ps, double *d, double *w1, double *w2, double *w3, double *w4,
                            double *w5, double *psn) {
    const size_t n = (size_t)H * W;
    const double c = P->c, a = P->a, a1 = P->a1, a2 = P->a2;
    const int eb = (P->algo == ORC_RPADMM_EB);
    const double rho = eb ? P->rho : 1.0;
    const double r = (P->algo == ORC_RPADMM_FG) ? P->r : 1.0;

    /* q_i^{k+1} = P_alpha((I - div^* div/a) q_i + grad(p_i - p_s - u_i/c)/a) */
    for (int i = 0; i < L; ++i) {
        double *Qx = qx + i * n, *Qy = qy + i * n;
        const double *Pi = p + i * n, *Ui = u + i * n;
        orc_div(H, W, Qx, Qy, w1);
        orc_div_adjoint(H, W, w1, w2, w3);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) w1[k] = Pi[k] - ps[k] - Ui[k] / c;
        orc_grad(H, W, w1, w4, w5);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            Qx[k] = Qx[k] - w2[k] / a + w4[k] / a;
            Qy[k] = Qy[k] - w3[k] / a + w5[k] / a;
        }
        orc_project_alpha(n, Qx, Qy, alpha, P->aniso);
        orc_div(H, W, Qx, Qy, d + i * n);
    }
    /* p_s^{k+1} (uses p^k and p_s^k) */
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        double s = 0.0;
        for (int i = 0; i < L; ++i) s += rho * d[i * n + k];
        for (int i = 0; i < L; ++i) s += rho * (p[i * n + k] - ps[k]) - u[i * n + k] / c;
        psn[k] = ps[k] + (s + 1.0 / c) / a2;
    }
    /* p_i^{k+1}, then u_i^{k+1} */
    for (int i = 0; i < L; ++i)
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            size_t ik = i * n + k;
            double p0 = p[ik];
            double p1 = dmin(p0 - (rho * (p0 - ps[k]) - u[ik] / c + rho * d[ik]) / a1, C[ik]);
            if (eb) {
                double newterm = P->literal_potts_u ? rho * (p1 - psn[k]) : (p1 - psn[k]);
                u[ik] = u[ik] - c * (rho * d[ik] + newterm - (1.0 - rho) * (p0 - ps[k]));
            } else {
                u[ik] = u[ik] - r * c * (d[ik] + p1 - psn[k]);
            }
            p[ik] = p1;
        }
    memcpy(ps, psn, n * sizeof(double));
}

/* One Potts pADMM-TY iteration (Eq. mADMM:Tai_yuan): the q_i-steps, then
 * the maximisations of the augmented Lagrangian over each p_i (with p_s^k)
 * and then over p_s (with the new p_i -- the sequential order the text after
 * the equation describes; the equation prints p_i^k), then the multiplier
 * steps u_i^{k+1} = u_i^k - c (p_i - p_s + div q_i)^{k+1}. */
static void potts_ty_step(int H, int W, int L, const double *C, const double *alpha,
                          const orc_params *P, double *u, double *qx, double *qy, double *p,
                          double *ps, double *d, double *w1, double *w2, double *w3, double *w4,
                          double *w5) {
    const size_t n = (size_t)H * W;
    const double c = P->c, a = P->a;
    for (int i = 0; i < L; ++i) {
        double *Qx = qx + i * n, *Qy = qy + i * n;
        const double *Pi = p + i * n, *Ui = u + i * n;
        orc_div(H, W, Qx, Qy, w1);
        orc_div_adjoint(H, W, w1, w2, w3);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) w1[k] = Pi[k] - ps[k] - Ui[k] / c;
        orc_grad(H, W, w1, w4, w5);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            Qx[k] = Qx[k] - w2[k] / a + w4[k] / a;
            Qy[k] = Qy[k] - w3[k] / a + w5[k] / a;
        }
        orc_project_alpha(n, Qx, Qy, alpha, P->aniso);
        orc_div(H, W, Qx, Qy, d + i * n);
    }
    for (int i = 0; i < L; ++i)
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            size_t ik = i * n + k;
            p[ik] = dmin(ps[k] - d[ik] + u[ik] / c, C[ik]);
        }
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        double s = 0.0;
        for (int i = 0; i < L; ++i) s += p[i * n + k] + d[i * n + k] - u[i * n + k] / c;
        ps[k] = s / L + 1.0 / (L * c);
    }
    for (int i = 0; i < L; ++i)
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            size_t ik = i * n + k;
            u[ik] = u[ik] - c * (p[ik] - ps[k] + d[ik]);
        }
}

/* One Potts rPDRQ iteration (Eq. pdrq:4labels, general L).  State (u_i,
 * qbar_i, pbar_i, pbar_s). */
static void potts_dr_step(int H, int W, int L, const double *C, const double *alpha,
                          const orc_params *P, double *u, double *qbx, double *qby, double *pb,
                          double *pbs, double *b, double *w1, double *w2, double *w3, double *w4,
                          double *usum) {
    const size_t n = (size_t)H * W;
    const double sg = P->sigma, tau = P->tau, rho = P->rho;
    /* b_i = -sigma (div qbar_i + pbar_i - pbar_s)
     *       + sigma tau ((L-1) u_i - sum_{j != i} u_j)   (uses u^k) */
    for (int i = 0; i < L; ++i) {
        orc_div(H, W, qbx + i * n, qby + i * n, b + i * n);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            double others = 0.0;
            for (int j = 0; j < L; ++j)
                if (j != i) others += u[j * n + k];
            b[i * n + k] = -sg * (b[i * n + k] + pb[i * n + k] - pbs[k]) +
                           sg * tau * ((L - 1) * u[i * n + k] - others);
        }
    }
    /* u_i^{k+1}: sRBGS for sigma tau T_0, T_0 = -Lap + (L+1) I (Lemma 1) */
    for (int i = 0; i < L; ++i) orc_srbgs(H, W, (double)(L + 1), sg * tau, b + i * n, u + i * n,
                                          P->sweeps);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        double s = 0.0;
        for (int i = 0; i < L; ++i) s += u[i * n + k];
        usum[k] = s;
    }
    for (int i = 0; i < L; ++i) {
        double *Ui = u + i * n, *Qx = qbx + i * n, *Qy = qby + i * n, *Pb = pb + i * n;
        const double *Ci = C + i * n;
        orc_grad(H, W, Ui, w1, w2);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            double q1 = Qx[k] - tau * w1[k];
            double q2 = Qy[k] - tau * w2[k];
            w3[k] = 2.0 * q1 - Qx[k];
            w4[k] = 2.0 * q2 - Qy[k];
            w1[k] = q1;
            w2[k] = q2;
        }
        orc_project_alpha(n, w3, w4, alpha, P->aniso);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            double p1 = Pb[k] + tau * Ui[k];
            Qx[k] = Qx[k] + rho * (w3[k] - w1[k]);
            Qy[k] = Qy[k] + rho * (w4[k] - w2[k]);
            Pb[k] = Pb[k] + rho * (dmin(2.0 * p1 - Pb[k], Ci[k]) - p1);
        }
    }
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        double ps1 = pbs[k] - tau * usum[k];
        pbs[k] = pbs[k] + rho * ((2.0 * ps1 - pbs[k] + tau) - ps1);
    }
}

/* ubar_i = u_i - tau (div q_i + p_i - p_s) (ALG1; see the readings above). */
static void potts_cp_ubar(int H, int W, int L, double tau, const double *u, const double *qx,
                          const double *qy, const double *p, const double *ps, double *ubar) {
    const size_t n = (size_t)H * W;
    for (int i = 0; i < L; ++i) {
        double *Ub = ubar + i * n;
        orc_div(H, W, qx + i * n, qy + i * n, Ub);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k)
            Ub[k] = u[i * n + k] - tau * (Ub[k] + p[i * n + k] - ps[k]);
    }
}

/* One Potts ALG1 iteration (Eq. alg1:4labels, general L): q_i, p_i and p_s
 * dual steps with ubar^k, the primal steps on u_i, ubar^{k+1} = 2u^{k+1} - u^k. */
static void potts_cp_step(int H, int W, int L, const double *C, const double *alpha,
                          const orc_params *P, double *u, double *qx, double *qy, double *p,
                          double *ps, double *ubar, double *w1, double *w2, double *w3) {
    const size_t n = (size_t)H * W;
    const double sg = P->sigma, tau = P->tau;
    for (int i = 0; i < L; ++i) {
        double *Qx = qx + i * n, *Qy = qy + i * n, *Pi = p + i * n;
        const double *Ub = ubar + i * n, *Ci = C + i * n;
        orc_grad(H, W, Ub, w1, w2);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            Qx[k] = Qx[k] - sg * w1[k];
            Qy[k] = Qy[k] - sg * w2[k];
        }
        orc_project_alpha(n, Qx, Qy, alpha, P->aniso);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) Pi[k] = dmin(Pi[k] + sg * Ub[k], Ci[k]);
    }
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        double s = 0.0;
        for (int i = 0; i < L; ++i) s += ubar[i * n + k];
        ps[k] = ps[k] - sg * s + sg;
    }
    for (int i = 0; i < L; ++i) {
        double *Ui = u + i * n, *Ub = ubar + i * n;
        orc_div(H, W, qx + i * n, qy + i * n, w3);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) {
            const double u0 = Ui[k];
            Ui[k] = u0 - tau * (w3[k] + p[i * n + k] - ps[k]);
            Ub[k] = 2.0 * Ui[k] - u0;
        }
    }
}

int orc_potts_run(int H, int W, int L, const double *C, const double *alpha, const orc_params *P,
                  int n_iter, int cold, double *u, double *qx, double *qy, double *p, double *ps) {
    if (P->algo < ORC_PADMM || P->algo > ORC_CP || L < 2 || L > 64) return -1;
    const size_t n = (size_t)H * W;
    if (cold) orc_potts_init(H, W, L, C, P->algo == ORC_RPDRQ, P->tau, u, qx, qy, p, ps);
    double *big = dalloc(n * L);
    double *w1 = dalloc(n), *w2 = dalloc(n), *w3 = dalloc(n), *w4 = dalloc(n), *w5 = dalloc(n),
           *w6 = dalloc(n);
    if (!big || !w1 || !w2 || !w3 || !w4 || !w5 || !w6) return -1;
    if (P->algo == ORC_CP) potts_cp_ubar(H, W, L, P->tau, u, qx, qy, p, ps, big);
    for (int it = 0; it < n_iter; ++it) {
        if (P->algo == ORC_CP)
            potts_cp_step(H, W, L, C, alpha, P, u, qx, qy, p, ps, big, w1, w2, w3);
        else if (P->algo == ORC_RPDRQ)
            potts_dr_step(H, W, L, C, alpha, P, u, qx, qy, p, ps, big, w1, w2, w3, w4, w6);
        else if (P->algo == ORC_TY)
            potts_ty_step(H, W, L, C, alpha, P, u, qx, qy, p, ps, big, w1, w2, w3, w4, w5);
        else
            potts_admm_step(H, W, L, C, alpha, P, u, qx, qy, p, ps, big, w1, w2, w3, w4, w5, w6);
    }
    free(big); free(w1); free(w2); free(w3); free(w4); free(w5); free(w6);
    return 0;
}

/* Certificates of the Potts state (out[0..3] = E, D, relative gap, l2
 * conservation residual over all labels).
 *  E(u) = sum_i sum_x ub_i C_i + alpha |grad ub_i|, ub(x) = projection of u(x)
 *         onto the simplex (Eq. relaxed-potts, Eq. pw-simplex).
 *  D(q) = sum_x min_i (C_i + div q_i) (Eq. potts-mf with p_s = p_i + div q_i).
 *  res  = || div q_i - p_s + p_i ||_2 over i and x.
 * For rPDRQ the flows are y = ybar + tau K u: q_i = qbar_i - tau grad u_i,
 * p_i = pbar_i + tau u_i, p_s = pbar_s - tau sum_i u_i; the dual uses
 * P_alpha(q_i). */
int orc_potts_eval(int H, int W, int L, const double *C, const double *alpha, int aniso, int dr,
                   double tau, const double *u, const double *qx, const double *qy,
                   const double *p, const double *ps, double *out) {
    if (L < 2 || L > 64) return -1; /* per-pixel label buffers hold 64 entries */
    const size_t n = (size_t)H * W;
    double *ub = dalloc(n * L), *gx = dalloc(n), *gy = dalloc(n), *fx = dalloc(n * L),
           *fy = dalloc(n * L), *fp = dalloc(n * L), *fs = dalloc(n), *d = dalloc(n),
           *mn = dalloc(n);
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        double v[64], w[64];
        for (int i = 0; i < L; ++i) v[i] = u[i * n + k];
        orc_simplex(L, v, w);
        for (int i = 0; i < L; ++i) ub[i * n + k] = w[i];
    }
    double E = 0.0;
    for (int i = 0; i < L; ++i) {
        orc_grad(H, W, ub + i * n, gx, gy);
        for (size_t k = 0; k < n; ++k) {
            double tv = aniso ? fabs(gx[k]) + fabs(gy[k]) : sqrt(gx[k] * gx[k] + gy[k] * gy[k]);
            E += ub[i * n + k] * C[i * n + k] + alpha[k] * tv;
        }
    }
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) {
        double s = 0.0;
        for (int i = 0; i < L; ++i) s += u[i * n + k];
        fs[k] = dr ? ps[k] - tau * s : ps[k];
    }
    for (int i = 0; i < L; ++i) {
        if (dr) {
            orc_grad(H, W, u + i * n, gx, gy);
            ORC_PAR_FOR(n)
            for (size_t k = 0; k < n; ++k) {
                fx[i * n + k] = qx[i * n + k] - tau * gx[k];
                fy[i * n + k] = qy[i * n + k] - tau * gy[k];
                fp[i * n + k] = p[i * n + k] + tau * u[i * n + k];
            }
        } else {
            memcpy(fx + i * n, qx + i * n, n * sizeof(double));
            memcpy(fy + i * n, qy + i * n, n * sizeof(double));
            memcpy(fp + i * n, p + i * n, n * sizeof(double));
        }
    }
    double res = 0.0;
    for (int i = 0; i < L; ++i) {
        orc_div(H, W, fx + i * n, fy + i * n, d);
        for (size_t k = 0; k < n; ++k) {
            double rr = d[k] - fs[k] + fp[i * n + k];
            res += rr * rr;
        }
    }
    ORC_PAR_FOR(n)
    for (size_t k = 0; k < n; ++k) mn[k] = INFINITY;
    for (int i = 0; i < L; ++i) {
        orc_project_alpha(n, fx + i * n, fy + i * n, alpha, aniso);
        orc_div(H, W, fx + i * n, fy + i * n, d);
        ORC_PAR_FOR(n)
        for (size_t k = 0; k < n; ++k) mn[k] = dmin(mn[k], C[i * n + k] + d[k]);
    }
    double D = 0.0;
    for (size_t k = 0; k < n; ++k) D += mn[k];
    out[0] = E;
    out[1] = D;
    out[2] = (E - D) / (fabs(E) > 1e-30 ? fabs(E) : 1e-30);
    out[3] = sqrt(res);
    free(ub); free(gx); free(gy); free(fx); free(fy); free(fp); free(fs); free(d); free(mn);
    return 0;
}
