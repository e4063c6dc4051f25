/*
 * oracle.h -- plain FP64 CPU oracle for the Crank-Nicolson step of the 3D time-dependent Dirac
 * equation in a dual-kinetic-balance B-spline x spherical-spinor basis (arXiv 2512.21697).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference arm may load, call or execute anything in oracle/.  The oracle shares no code,
 * header, table or constant with the CUDA library; the two are built separately and neither
 * includes nor links the other.
 *
 * Everything here is double precision (the paper computes in double-precision complex, Sec. 4).
 * Complex vectors are arrays of interleaved (re, im) doubles.
 *
 * Vector layout ("paper order"): channel-major; channel c owns 2(N+1) consecutive coefficients,
 * the first N+1 of the "large" DKB type (P = u_k) and the next N+1 of the "small" type (Q = u_k),
 * Eq. (dualkinetic), built on B-splines B_1 .. B_{N+1} of the full knot vector B_0 .. B_{N+3}.
 * B_1 is used only where both DKB components vanish at r = 0 (large type for kappa = -1, small
 * type for kappa = +1); the unused coefficients stay zero and the operators act on them as the
 * identity.  Channels are enumerated kappa = -1, 1, -2, 2, ... and, inside one kappa,
 * 2mu ascending.
 */
#ifndef DIRAC_ORACLE_H
#define DIRAC_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double Z, c, R;      /* nuclear charge, speed of light (a.u.), box radius                    */
    int N;               /* retained B-splines per radial block                                  */
    int order;           /* B-spline order k (polynomial degree k-1)                             */
    int grid;            /* 0 linear breakpoints, 1 linear up to r_lin then geometric,           */
                         /* 2 exponential: first interval r_lin, ratio fixed by the last = R     */
    double r_lin;        /* grid 1: end of the linear part; grid 2: the first interval           */
    int n_lin;           /* grid 1: number of linear intervals                                   */
    int kappa_max;       /* |kappa| <= kappa_max                                                 */
    int two_mu_max;      /* |2mu| <= two_mu_max; <= 0 keeps every mu                             */
    int l_max;           /* multipole truncation of the plane-wave expansion                     */
    int quad;            /* Gauss-Legendre points per knot interval                              */
    double E0, omega, n_cycles; /* sin^2 pulse, Eq. (ndpPot)                                     */
    double dt;           /* time step                                                            */
    int time_eval;       /* 0: H at t+dt/2 (midpoint rule), 1: H at t+dt (Eq. solPsi as printed) */
    int b1_drop;         /* 1: the literal boundary reading, B_1 removed for every kappa too      */
} or_params;

typedef struct or_ctx or_ctx;

or_ctx* or_create(const or_params* p);
void    or_free(or_ctx* c);
int     or_nchannels(const or_ctx* c);
void    or_channels(const or_ctx* c, int* kappa, int* two_mu);
int     or_nknots(const or_ctx* c);
void    or_knots(const or_ctx* c, double* out);
int     or_nedges(or_ctx* c);                 /* ordered coupled channel pairs               */
void    or_edges(or_ctx* c, int* a, int* b);

/* B-splines (Sec. 2.2): all N+4 splines of the full knot vector at x, with 1st/2nd derivative. */
void   or_bspline_all(const or_ctx* c, double x, double* val, double* d1, double* d2);
void   or_gauss_legendre(int q, double* x, double* w);
/* Radial blocks for one kappa (2(N+1) x 2(N+1), paper order, row-major). */
void   or_radial_dense(or_ctx* c, int kappa, double* S, double* H0);
void   or_radial_rmoment(or_ctx* c, int kappa, double* Rm);
/* Spherical spinor X_{kappa,mu}(theta,phi) (2 complex components). */
void   or_spinor(int kappa, int two_mu, double theta, double phi, double* out4);
double or_angular(int kappa1, int two_mu1, int kappa2, int two_mu2, int l);
double or_angular_2d(int kappa1, int two_mu1, int kappa2, int two_mu2, int l, int nth, int nph);
double or_sph_bessel(int l, double x);
double or_field_direct(const or_ctx* c, double t, double r, double cos_theta);
double or_field_series(const or_ctx* c, double t, double r, double cos_theta, int lmax);
double or_field_F(const or_ctx* c, double t, double r, int l);
/* Coupling block X_ab(t) (real, 2(N+1) square): H_ab = i X_ab, ordered channels a != b. */
void   or_coupling_block(or_ctx* c, int a, int b, double t, double* X);
/* Brute-force <psi_{a,i}| H_I(t) |psi_{b,j}> by 3D quadrature with the untruncated pulse. */
void   or_coupling_3d(or_ctx* c, int a, int i, int b, int j, double t, int nth, int nph, double* out2);
/* y = A_sign(t) x with A_+- = S +- i tau H(t), tau = dt/2; t is the evaluation time of H. */
void   or_apply(or_ctx* c, double t, int sign, const double* x, double* y);
void   or_apply_rows(or_ctx* c, double t, int sign, const double* x, int nrows,
                     const int* ch, const int* idx, double* out);
/* Dense A_sign(t) (n x n complex) for tiny bases. */
void   or_dense_operator(or_ctx* c, double t, int sign, double* A);
int    or_dense_solve(int n, const double* A, const double* b, double* x);
void   or_precond(or_ctx* c, const double* r, double* z);
/* One Crank-Nicolson step from t_n: psi <- A_+^{-1} A_- psi.  Returns BiCGSTAB iterations or <0. */
int    or_step(or_ctx* c, double* psi, double t_n, double tol, int max_iter, int precond,
               double* resid_out);
int    or_step_dense(or_ctx* c, double* psi, double t_n);
/* Generalised eigenproblem H0 v = E S v for one kappa, ascending, v^T S v = 1.  E and V (rows)
 * have room for 2(N+1) pairs; returns the number of basis functions this kappa uses (the rest of
 * E is +inf and the rest of V zero). */
int    or_eigen(or_ctx* c, int kappa, double* E, double* V);
/* norm, <H0>, P_ground, P_bound */
void   or_observables(or_ctx* c, const double* psi, double* out4);

#ifdef __cplusplus
}
#endif
#endif
