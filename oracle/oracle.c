/*
 * oracle.c -- plain FP64 CPU oracle of the Crank-Nicolson step of the 3D time-dependent Dirac
 * equation (arXiv 2512.21697, "GaDE"), written from the paper's equations.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference arm may load or run it.  It shares no code with the CUDA library.
 *
 * The oracle computes the *definition* of each quantity, slowly:
 *   - B-splines by the Cox-de Boor recursion (Sec. 2.2), evaluated over the whole knot vector;
 *   - DKB radial functions (Eq. dualkinetic) and the radial matrix elements of H0 and S computed
 *     directly for the actual kappa (no kappa-polynomial split);
 *   - angular coefficients <X_{k1 m1}| sigma_x (2l+1) P_l(cos th) |X_{k2 m2}> (Eq. Htheta,
 *     4 pi Y_l0(z) Y_l0(r) = (2l+1) P_l(cos th)) by Gauss-Legendre quadrature in cos(theta) with the
 *     phi integral done by orthogonality of e^{i m phi} (no Clebsch-Gordan x 3j route);
 *   - the pulse (Eq. ndpPot) through its separable plane-wave form (Eq. bdpA), each multipole l
 *     summed over the three sin^2 carriers directly at the quadrature points;
 *   - the interaction matrix element of H_I = -c alpha.A (Eq. interactionH) between the 4-spinor
 *     basis functions of Eq. (basis), reduced to radial x angular integrals;
 *   - the Crank-Nicolson propagator of Eq. (solPsi) solved by its own right-preconditioned
 *     BiCGSTAB (preconditioner: dense LU of M = S + i dt/2 H0, Eq. matrixM) and, for tiny
 *     bases, by a dense LU solve.
 *
 * Readings of the paper where it is silent or garbled:
 *   - p = -i grad (the printed "p = i grad" is a sign slip; with -i grad the DKB pairing of
 *     Eq. dualkinetic is the kinetic-balance one and no spurious states appear).
 *   - alpha_i = [[0, sigma_i], [sigma_i, 0]] (the printed lower block "-sigma_i" is not Hermitian).
 *   - The lower spinor of the basis is i Q X_{-kappa,mu} (Eq. basis); the matrix-element print
 *     that repeats X_{kappa} in the lower row is a typo.
 *   - V(r) in "-I_4 V(r)" is the attractive Coulomb potential Z/r, so the potential energy is -Z/r.
 *   - "Degree d = 7" is read as B-spline order k (the order is a parameter here).
 *   - The first two and the last two B-splines are removed (zero value and first derivative at
 *     r = 0, "a similar choice" at r_max).  B_1, the first one kept, is nonzero in slope at r = 0;
 *     it is used only where both radial components of the DKB pair still vanish there: the large
 *     type of kappa = -1 (P = B_1, Q = (B_1' - B_1/r)/2c, both zero at r = 0) and the small type of
 *     kappa = +1; every other slot built on B_1 is left out (identity in S, zero in H).  Without it
 *     the 1s level misses its closed form.  The literal reading (B_1 removed everywhere) is the
 *     b1_drop = 1 option; on knots refined towards r = 0 (grid 2) its 1s miss falls only slowly,
 *     to 1e-3 with a first interval of 1e-5, against ~1e-11 with B_1 kept as above.
 *   - Polarisation x, propagation z (sigma_x and Y_l0(z) in Eq. Htheta).  The pulse is switched
 *     on for 0 <= t <= T globally and its separable form is used at every r inside that window.
 *   - H(t) in a step is taken at the midpoint t + dt/2 (the derivation of Sec. 2.4); the printed
 *     H(t + dt) of Eq. solPsi is the time_eval = 1 option.
 *   - The LU of M (Eq. matrixM) uses partial pivoting (M is complex symmetric, not Hermitian);
 *     the preconditioner changes iteration counts only, never the converged step.
 *   - The stopping test is the true relative residual ||b - A_+ x||_2 <= tol ||b||_2, BiCGSTAB
 *     right-preconditioned with shadow vector r0.
 */
#include "oracle.h"
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define MAXL 64

struct edge_info {
    int b;          /* neighbour channel */
    double* A1;     /* A1_l = a_l(kappa_a, mu_a; -kappa_b, mu_b), l = 0..l_max */
    double* A2;     /* A2_l = a_l(-kappa_a, mu_a; kappa_b, mu_b)               */
};

struct or_ctx {
    or_params p;
    int m;              /* breakpoint intervals              */
    int nsp;            /* N + 4 B-splines                   */
    int nk;             /* knots = nsp + order               */
    double* t;          /* knot vector                       */
    double* brk;        /* m + 1 breakpoints                 */
    int npts;
    double *pr, *pw;    /* quadrature points / weights       */
    int* pint;          /* interval of each point            */
    double *bv, *bd, *bdd; /* [npts][order]: splines pint..pint+order-1 */
    double T, Om, w[3], wt[3];
    double* jl;         /* [3][l_max+1][npts] spherical Bessel j_l(w_c r / c) */
    int nch;
    int *kap, *tmu;
    /* per-kappa dense radial blocks (small bases only) */
    double **S, **H;
    cplx** Mlu;
    int** Mpiv;
    double **E, **V;    /* eigen decompositions */
    /* adjacency (lazily built per channel) */
    int* adj_done;
    int* nadj;
    struct edge_info** adj;
    /* dense coupling blocks at one time (small bases only) */
    double cache_t;
    int cache_ok;
    double*** X;        /* X[a][e] for e-th neighbour of a */
};

/* ------------------------------------------------------------------------------------------ */
/* Small helpers                                                                               */
/* ------------------------------------------------------------------------------------------ */

static int lkap(int kappa) { return kappa > 0 ? kappa : -kappa - 1; }
static int kslot(int kappa) { return 2 * (abs(kappa) - 1) + (kappa > 0 ? 1 : 0); }
static int nkslots(const or_ctx* c) { return 2 * c->p.kappa_max; }
static int nslot(const or_ctx* c) { return c->p.N + 1; }
static int dim2(const or_ctx* c) { return 2 * nslot(c); }

/* Basis function i of a channel: i < N+1 is the large DKB type built on spline B_{i+1},
 * i >= N+1 the small type built on B_{i-N} (full-knot-vector numbering B_0 .. B_{N+3}).
 * The zero boundary condition P(0) = Q(0) = 0 (Sec. 2.2) removes B_0 (nonzero at 0) and every
 * DKB function whose components do not vanish at 0.  B_1 ~ r keeps P(0) = Q(0) = 0 only as the
 * large type for kappa = -1 (Q = (u' - u/r)/2c) and as the small type for kappa = +1
 * (P = (u' - u/r)/2c); B_{N+2}, B_{N+3} break the condition at r_max and are removed. */
static int active(const or_ctx* c, int kappa, int i)
{
    if (i == 0) return !c->p.b1_drop && kappa == -1;
    if (i == nslot(c)) return !c->p.b1_drop && kappa == 1;
    return 1;
}

static int find_channel(const or_ctx* c, int kappa, int two_mu)
{
    for (int a = 0; a < c->nch; a++)
        if (c->kap[a] == kappa && c->tmu[a] == two_mu) return a;
    return -1;
}

/* ------------------------------------------------------------------------------------------ */
/* Knots (Sec. 2.2): order-fold end knots; linear breakpoints, or linear then geometric.       */
/* ------------------------------------------------------------------------------------------ */

static void make_breakpoints(or_ctx* c)
{
    const or_params* p = &c->p;
    int m = c->m;
    c->brk = (double*)malloc(sizeof(double) * (m + 1));
    if (p->grid == 1 && p->n_lin > 0 && p->n_lin < m && p->r_lin < p->R) {
        double h = p->r_lin / p->n_lin;
        int M = m - p->n_lin;
        double rest = p->R - p->r_lin;
        /* gamma solves h * sum_{i=1..M} gamma^i = R - r_lin (bisection). */
        double lo = 1.0, hi = 2.0;
        for (;;) {
            double s = 0, g = 1;
            for (int i = 1; i <= M; i++) { g *= hi; s += g; }
            if (h * s > rest) break;
            hi *= 2;
        }
        for (int it = 0; it < 200; it++) {
            double mid = 0.5 * (lo + hi), s = 0, g = 1;
            for (int i = 1; i <= M; i++) { g *= mid; s += g; }
            if (h * s > rest) hi = mid; else lo = mid;
        }
        double gam = 0.5 * (lo + hi);
        for (int i = 0; i <= p->n_lin; i++) c->brk[i] = h * i;
        double r = p->r_lin, g = 1;
        for (int j = 1; j <= M; j++) { g *= gam; r += h * g; c->brk[p->n_lin + j] = r; }
        c->brk[m] = p->R;
    } else if (p->grid == 2 && p->r_lin > 0 && p->r_lin * m < p->R) {
        /* r_i = h (g^i - 1) / (g - 1), g > 1 by bisection so that r_m = R (knots dense near r = 0) */
        double h = p->r_lin, lo = 1.0, hi = 2.0;
        while (h * (pow(hi, m) - 1.0) / (hi - 1.0) < p->R) hi *= 2.0;
        for (int it = 0; it < 200; it++) {
            double mid = 0.5 * (lo + hi);
            if (h * (pow(mid, m) - 1.0) / (mid - 1.0) > p->R) hi = mid; else lo = mid;
        }
        double g = 0.5 * (lo + hi);
        for (int i = 0; i <= m; i++) c->brk[i] = h * (pow(g, i) - 1.0) / (g - 1.0);
        c->brk[m] = p->R;
    } else {
        for (int i = 0; i <= m; i++) c->brk[i] = p->R * (double)i / (double)m;
    }
}

static void make_knots(or_ctx* c)
{
    int k = c->p.order;
    c->t = (double*)malloc(sizeof(double) * c->nk);
    for (int i = 0; i < k - 1; i++) c->t[i] = 0.0;
    for (int i = 0; i <= c->m; i++) c->t[k - 1 + i] = c->brk[i];
    for (int i = 0; i < k - 1; i++) c->t[k + c->m + i] = c->p.R;
}

/* ------------------------------------------------------------------------------------------ */
/* Cox-de Boor recursion (Sec. 2.2), whole knot vector, degree 0..k-1.                         */
/* u_{s,0}(x) = 1 on t_s < x <= t_{s+1};                                                       */
/* u_{s,d} = (x-t_s)/(t_{s+d}-t_s) u_{s,d-1} + (t_{s+d+1}-x)/(t_{s+d+1}-t_{s+1}) u_{s+1,d-1}.  */
/* Derivatives: D u_{s,d} = d (u_{s,d-1}/(t_{s+d}-t_s) - u_{s+1,d-1}/(t_{s+d+1}-t_{s+1})).    */
/* ------------------------------------------------------------------------------------------ */

static double safe_div(double a, double b) { return b > 0 ? a / b : 0.0; }

static void bspline_table(const double* t, int nk, int k, double x, double* B /* k*nk */)
{
    for (int i = 0; i < k * nk; i++) B[i] = 0;
    for (int s = 0; s < nk - 1; s++) B[s] = (t[s] < x && x <= t[s + 1]) ? 1.0 : 0.0;
    for (int d = 1; d < k; d++)
        for (int s = 0; s < nk - 1 - d; s++) {
            double a = safe_div(x - t[s], t[s + d] - t[s]) * B[(d - 1) * nk + s];
            double b = safe_div(t[s + d + 1] - x, t[s + d + 1] - t[s + 1]) * B[(d - 1) * nk + s + 1];
            B[d * nk + s] = a + b;
        }
}

static void bspline_eval(const double* t, int nk, int k, double x, double* val, double* d1, double* d2)
{
    int ns = nk - k;
    double* B = (double*)malloc(sizeof(double) * k * nk);
    bspline_table(t, nk, k, x, B);
    int d = k - 1;
    for (int s = 0; s < ns; s++) {
        val[s] = B[d * nk + s];
        /* first derivative of the degree-d spline */
        d1[s] = d * (safe_div(B[(d - 1) * nk + s], t[s + d] - t[s]) -
                     safe_div(B[(d - 1) * nk + s + 1], t[s + d + 1] - t[s + 1]));
        /* second derivative: the same formula applied to the degree-(d-1) derivatives */
        double e0 = (d - 1) * (safe_div(B[(d - 2) * nk + s], t[s + d - 1] - t[s]) -
                               safe_div(B[(d - 2) * nk + s + 1], t[s + d] - t[s + 1]));
        double e1 = (d - 1) * (safe_div(B[(d - 2) * nk + s + 1], t[s + d] - t[s + 1]) -
                               safe_div(B[(d - 2) * nk + s + 2], t[s + d + 1] - t[s + 2]));
        d2[s] = d * (safe_div(e0, t[s + d] - t[s]) - safe_div(e1, t[s + d + 1] - t[s + 1]));
    }
    free(B);
}

void or_bspline_all(const or_ctx* c, double x, double* val, double* d1, double* d2)
{
    bspline_eval(c->t, c->nk, c->p.order, x, val, d1, d2);
}

/* ------------------------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [-1,1]: Newton iteration on P_q via the three-term recurrence.      */
/* ------------------------------------------------------------------------------------------ */

void or_gauss_legendre(int q, double* x, double* w)
{
    for (int i = 0; i < q; i++) {
        double z = cos(M_PI * (i + 0.75) / (q + 0.5)), dp = 0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1, p1 = z;
            for (int n = 2; n <= q; n++) {
                double p2 = ((2 * n - 1) * z * p1 - (n - 1) * p0) / n;
                p0 = p1; p1 = p2;
            }
            if (q == 1) { p1 = z; p0 = 1; }
            dp = q * (z * p1 - p0) / (z * z - 1);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1, p1 = z;
        for (int n = 2; n <= q; n++) {
            double p2 = ((2 * n - 1) * z * p1 - (n - 1) * p0) / n;
            p0 = p1; p1 = p2;
        }
        if (q == 1) { p1 = z; p0 = 1; }
        dp = q * (z * p1 - p0) / (z * z - 1);
        x[i] = z;
        w[i] = 2.0 / ((1 - z * z) * dp * dp);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Spherical Bessel j_l by its power series j_l(x) = x^l sum_k (-x^2/2)^k / (k! (2l+2k+1)!!). */
/* ------------------------------------------------------------------------------------------ */

double or_sph_bessel(int l, double x)
{
    double df = 1.0; /* (2l+1)!! */
    for (int i = 3; i <= 2 * l + 1; i += 2) df *= i;
    double term = pow(x, l) / df, sum = term;
    for (int kk = 1; kk < 400; kk++) {
        term *= -0.5 * x * x / (kk * (2.0 * l + 2.0 * kk + 1.0));
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum)) break;
    }
    return sum;
}

/* ------------------------------------------------------------------------------------------ */
/* Context                                                                                     */
/* ------------------------------------------------------------------------------------------ */

or_ctx* or_create(const or_params* p)
{
    if (p->order < 3 || p->N < 1 || p->kappa_max < 1 || p->quad < 1 || p->l_max < 0 ||
        p->l_max >= MAXL)
        return NULL;
    or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
    c->p = *p;
    int k = p->order;
    c->nsp = p->N + 4;
    c->m = c->nsp - k + 1;
    if (c->m < 1) { free(c); return NULL; }
    c->nk = c->nsp + k;
    make_breakpoints(c);
    make_knots(c);

    /* quadrature points: q Gauss-Legendre nodes per breakpoint interval */
    int q = p->quad;
    double* gx = (double*)malloc(sizeof(double) * q);
    double* gw = (double*)malloc(sizeof(double) * q);
    or_gauss_legendre(q, gx, gw);
    c->npts = c->m * q;
    c->pr = (double*)malloc(sizeof(double) * c->npts);
    c->pw = (double*)malloc(sizeof(double) * c->npts);
    c->pint = (int*)malloc(sizeof(int) * c->npts);
    c->bv = (double*)malloc(sizeof(double) * c->npts * k);
    c->bd = (double*)malloc(sizeof(double) * c->npts * k);
    c->bdd = (double*)malloc(sizeof(double) * c->npts * k);
    double* v = (double*)malloc(sizeof(double) * c->nsp);
    double* d1 = (double*)malloc(sizeof(double) * c->nsp);
    double* d2 = (double*)malloc(sizeof(double) * c->nsp);
    for (int i = 0; i < c->m; i++) {
        double a = c->brk[i], b = c->brk[i + 1];
        for (int j = 0; j < q; j++) {
            int pp = i * q + j;
            double x = 0.5 * (a + b) + 0.5 * (b - a) * gx[j];
            c->pr[pp] = x;
            c->pw[pp] = 0.5 * (b - a) * gw[j];
            c->pint[pp] = i;
            bspline_eval(c->t, c->nk, k, x, v, d1, d2);
            for (int s = 0; s < k; s++) {
                int tot = i + s;
                c->bv[pp * k + s] = tot < c->nsp ? v[tot] : 0;
                c->bd[pp * k + s] = tot < c->nsp ? d1[tot] : 0;
                c->bdd[pp * k + s] = tot < c->nsp ? d2[tot] : 0;
            }
        }
    }
    free(v); free(d1); free(d2); free(gx); free(gw);

    /* pulse carriers: sin^2(pi s/T) sin(w s) = 1/2 sin(w s) - 1/4 sin((w+Om)s) - 1/4 sin((w-Om)s) */
    c->T = p->n_cycles * 2 * M_PI / p->omega;
    c->Om = 2 * M_PI / c->T;
    c->w[0] = p->omega;           c->wt[0] = 0.5;
    c->w[1] = p->omega + c->Om;   c->wt[1] = -0.25;
    c->w[2] = p->omega - c->Om;   c->wt[2] = -0.25;
    int L = p->l_max + 1;
    c->jl = (double*)malloc(sizeof(double) * 3 * L * c->npts);
    for (int cc = 0; cc < 3; cc++)
        for (int l = 0; l < L; l++)
            for (int pp = 0; pp < c->npts; pp++)
                c->jl[(cc * L + l) * c->npts + pp] = or_sph_bessel(l, c->w[cc] * c->pr[pp] / p->c);

    /* channels */
    int cap = 0;
    for (int ak = 1; ak <= p->kappa_max; ak++) cap += 2 * 2 * ak;
    c->kap = (int*)malloc(sizeof(int) * cap);
    c->tmu = (int*)malloc(sizeof(int) * cap);
    c->nch = 0;
    for (int ak = 1; ak <= p->kappa_max; ak++)
        for (int sg = -1; sg <= 1; sg += 2) {
            int kappa = sg * ak;
            for (int tm = -(2 * ak - 1); tm <= 2 * ak - 1; tm += 2)
                if (p->two_mu_max <= 0 || abs(tm) <= p->two_mu_max) {
                    c->kap[c->nch] = kappa;
                    c->tmu[c->nch] = tm;
                    c->nch++;
                }
        }
    int ns = nkslots(c);
    c->S = (double**)calloc(ns, sizeof(double*));
    c->H = (double**)calloc(ns, sizeof(double*));
    c->Mlu = (cplx**)calloc(ns, sizeof(cplx*));
    c->Mpiv = (int**)calloc(ns, sizeof(int*));
    c->E = (double**)calloc(ns, sizeof(double*));
    c->V = (double**)calloc(ns, sizeof(double*));
    c->adj_done = (int*)calloc(c->nch, sizeof(int));
    c->nadj = (int*)calloc(c->nch, sizeof(int));
    c->adj = (struct edge_info**)calloc(c->nch, sizeof(struct edge_info*));
    c->X = (double***)calloc(c->nch, sizeof(double**));
    c->cache_ok = 0;
    return c;
}

static void drop_coupling_cache(or_ctx* c)
{
    for (int a = 0; a < c->nch; a++) {
        if (!c->X[a]) continue;
        for (int e = 0; e < c->nadj[a]; e++) free(c->X[a][e]);
        free(c->X[a]);
        c->X[a] = NULL;
    }
    c->cache_ok = 0;
}

void or_free(or_ctx* c)
{
    if (!c) return;
    drop_coupling_cache(c);
    for (int s = 0; s < nkslots(c); s++) {
        free(c->S[s]); free(c->H[s]); free(c->Mlu[s]); free(c->Mpiv[s]); free(c->E[s]); free(c->V[s]);
    }
    for (int a = 0; a < c->nch; a++) {
        for (int e = 0; e < c->nadj[a]; e++) { free(c->adj[a][e].A1); free(c->adj[a][e].A2); }
        free(c->adj[a]);
    }
    free(c->S); free(c->H); free(c->Mlu); free(c->Mpiv); free(c->E); free(c->V);
    free(c->adj); free(c->adj_done); free(c->nadj); free(c->X);
    free(c->t); free(c->brk); free(c->pr); free(c->pw); free(c->pint);
    free(c->bv); free(c->bd); free(c->bdd); free(c->jl); free(c->kap); free(c->tmu);
    free(c);
}

int or_nchannels(const or_ctx* c) { return c->nch; }
void or_channels(const or_ctx* c, int* kappa, int* two_mu)
{
    memcpy(kappa, c->kap, sizeof(int) * c->nch);
    memcpy(two_mu, c->tmu, sizeof(int) * c->nch);
}
int or_nknots(const or_ctx* c) { return c->nk; }
void or_knots(const or_ctx* c, double* out) { memcpy(out, c->t, sizeof(double) * c->nk); }

/* ------------------------------------------------------------------------------------------ */
/* Dual kinetic balance functions (Eq. dualkinetic) at quadrature point pp.                    */
/* large type (i < N+1): P = u, Q = (u' + kappa u / r) / 2c                                    */
/* small type (i >= N+1): P = (u' - kappa u / r) / 2c, Q = u                                   */
/* u = B_{(i mod (N+1)) + 1}; unused functions (see active()) are identically zero.            */
/* ------------------------------------------------------------------------------------------ */

static int dkb(const or_ctx* c, int pp, int kappa, int i, double* P, double* dP, double* Q, double* dQ)
{
    int N1 = nslot(c), k = c->p.order;
    int s = (i % N1) + 1;
    int j = s - c->pint[pp];
    if (j < 0 || j >= k || !active(c, kappa, i)) { *P = *dP = *Q = *dQ = 0; return 0; }
    double u = c->bv[pp * k + j], du = c->bd[pp * k + j], ddu = c->bdd[pp * k + j];
    double r = c->pr[pp], tc = 2 * c->p.c;
    if (i < N1) {
        *P = u; *dP = du;
        *Q = (du + kappa * u / r) / tc;
        *dQ = (ddu + kappa * (du / r - u / (r * r))) / tc;
    } else {
        *P = (du - kappa * u / r) / tc;
        *dP = (ddu - kappa * (du / r - u / (r * r))) / tc;
        *Q = u; *dQ = du;
    }
    return 1;
}

/* point range where the splines of basis i and basis j overlap; returns 0 if disjoint */
static int common_points(const or_ctx* c, int i, int j, int* p0, int* p1)
{
    int N1 = nslot(c), k = c->p.order, q = c->p.quad;
    int si = (i % N1) + 1, sj = (j % N1) + 1;
    int lo = (si > sj ? si : sj) - k + 1, hi = si < sj ? si : sj;
    if (lo < 0) lo = 0;
    if (hi > c->m - 1) hi = c->m - 1;
    if (lo > hi) return 0;
    *p0 = lo * q;
    *p1 = (hi + 1) * q;
    return 1;
}

/* ------------------------------------------------------------------------------------------ */
/* Radial matrix elements for one kappa (Eq. TDDE with H0 = beta c^2 - V + c alpha.p):        */
/*   S_ij  = int (P_i P_j + Q_i Q_j) dr                                                        */
/*   H0_ij = int [ P_i U P_j + Q_i (U - 2c^2) Q_j - c P_i (Q_j' - kappa Q_j / r)              */
/*                 + c Q_i (P_j' + kappa P_j / r) ] dr,     U = -Z / r                          */
/* obtained from (sigma.p) [f(r)/r X_{kappa mu}] = (i/r)(f' + kappa f / r) X_{-kappa mu}.      */
/* ------------------------------------------------------------------------------------------ */

static void radial_elem(const or_ctx* c, int kappa, int i, int j, double* s_out, double* h_out)
{
    int p0, p1;
    double s = 0, h = 0;
    if (common_points(c, i, j, &p0, &p1)) {
        double cc = c->p.c, Z = c->p.Z;
        for (int pp = p0; pp < p1; pp++) {
            double Pi, dPi, Qi, dQi, Pj, dPj, Qj, dQj;
            dkb(c, pp, kappa, i, &Pi, &dPi, &Qi, &dQi);
            dkb(c, pp, kappa, j, &Pj, &dPj, &Qj, &dQj);
            double r = c->pr[pp], w = c->pw[pp], U = -Z / r;
            s += w * (Pi * Pj + Qi * Qj);
            h += w * (Pi * U * Pj + Qi * (U - 2 * cc * cc) * Qj - cc * Pi * (dQj - kappa * Qj / r) +
                      cc * Qi * (dPj + kappa * Pj / r));
        }
    }
    *s_out = s;
    *h_out = h;
}

static void ensure_radial(or_ctx* c, int kappa)
{
    int sl = kslot(kappa), n = dim2(c);
    if (c->S[sl]) return;
    double* S = (double*)calloc((size_t)n * n, sizeof(double));
    double* H = (double*)calloc((size_t)n * n, sizeof(double));
    #pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) radial_elem(c, kappa, i, j, &S[(size_t)i * n + j], &H[(size_t)i * n + j]);
    c->S[sl] = S;
    c->H[sl] = H;
}

void or_radial_dense(or_ctx* c, int kappa, double* S, double* H0)
{
    int n = dim2(c);
    ensure_radial(c, kappa);
    memcpy(S, c->S[kslot(kappa)], sizeof(double) * n * n);
    memcpy(H0, c->H[kslot(kappa)], sizeof(double) * n * n);
}

void or_radial_rmoment(or_ctx* c, int kappa, double* Rm)
{
    int n = dim2(c);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            int p0, p1;
            double s = 0;
            if (common_points(c, i, j, &p0, &p1))
                for (int pp = p0; pp < p1; pp++) {
                    double Pi, dPi, Qi, dQi, Pj, dPj, Qj, dQj;
                    dkb(c, pp, kappa, i, &Pi, &dPi, &Qi, &dQi);
                    dkb(c, pp, kappa, j, &Pj, &dPj, &Qj, &dQj);
                    s += c->pw[pp] * c->pr[pp] * (Pi * Pj + Qi * Qj);
                }
            Rm[(size_t)i * n + j] = s;
        }
}

/* ------------------------------------------------------------------------------------------ */
/* Spherical spinors (Eq. spinorbasis) with the spin-1/2 Clebsch-Gordan closed forms:          */
/*  j = l + 1/2 (kappa < 0): C_up = sqrt((l+mu+1/2)/(2l+1)),  C_dn = sqrt((l-mu+1/2)/(2l+1))    */
/*  j = l - 1/2 (kappa > 0): C_up = -sqrt((l-mu+1/2)/(2l+1)), C_dn = sqrt((l+mu+1/2)/(2l+1))    */
/* X = (C_up Y_{l,mu-1/2}, C_dn Y_{l,mu+1/2}); Y_lm with the Condon-Shortley phase.            */
/* ------------------------------------------------------------------------------------------ */

static void spinor_cg(int kappa, int two_mu, double* cu, double* cd)
{
    int l = lkap(kappa);
    double mu = 0.5 * two_mu, d = 2.0 * l + 1.0;
    double a = (l + mu + 0.5) / d, b = (l - mu + 0.5) / d;
    if (a < 0) a = 0;
    if (b < 0) b = 0;
    if (kappa < 0) { *cu = sqrt(a); *cd = sqrt(b); }
    else { *cu = -sqrt(b); *cd = sqrt(a); }
}

/* P_l^m(x), m >= 0, Condon-Shortley phase included */
static double assoc_legendre(int l, int m, double x)
{
    if (m < 0 || m > l) return 0.0;
    double pmm = 1.0, s = sqrt(fmax(0.0, (1 - x) * (1 + x)));
    for (int i = 1; i <= m; i++) pmm *= -(2.0 * i - 1.0) * s;
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double pl = 0;
    for (int ll = m + 2; ll <= l; ll++) {
        pl = (x * (2.0 * ll - 1.0) * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pm1;
        pm1 = pl;
    }
    return pl;
}

/* theta part of Y_lm: Y_lm(theta,phi) = Theta_lm(cos theta) e^{i m phi} */
static double theta_lm(int l, int m, double x)
{
    int am = abs(m);
    if (am > l) return 0.0;
    double nrm = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * exp(lgamma(l - am + 1.0) - lgamma(l + am + 1.0)));
    double v = nrm * assoc_legendre(l, am, x);
    if (m < 0 && (am & 1)) v = -v;
    return v;
}

static double legendre(int l, double x) { return assoc_legendre(l, 0, x); }

void or_spinor(int kappa, int two_mu, double theta, double phi, double* out4)
{
    int l = lkap(kappa);
    double cu, cd;
    spinor_cg(kappa, two_mu, &cu, &cd);
    int mu_up = (two_mu - 1) / 2, mu_dn = (two_mu + 1) / 2;
    double x = cos(theta);
    cplx up = cu * theta_lm(l, mu_up, x) * cexp(I * mu_up * phi);
    cplx dn = cd * theta_lm(l, mu_dn, x) * cexp(I * mu_dn * phi);
    out4[0] = creal(up); out4[1] = cimag(up);
    out4[2] = creal(dn); out4[3] = cimag(dn);
}

/* 2 pi int_{-1}^{1} Theta_{l1 m}(x) Theta_{l2 m}(x) (2l+1) P_l(x) dx, exact Gauss-Legendre */
static double theta_integral(int l1, int l2, int m, int l)
{
    int n = (l1 + l2 + l) / 2 + 2;
    double* x = (double*)malloc(sizeof(double) * n);
    double* w = (double*)malloc(sizeof(double) * n);
    or_gauss_legendre(n, x, w);
    double s = 0;
    for (int i = 0; i < n; i++) s += w[i] * theta_lm(l1, m, x[i]) * theta_lm(l2, m, x[i]) * (2 * l + 1) * legendre(l, x[i]);
    free(x); free(w);
    return 2 * M_PI * s;
}

/* a_l(k1,m1; k2,m2) = int dOmega X_{k1 m1}^dagger sigma_x (2l+1) P_l(cos th) X_{k2 m2}
 *                   = <X_{k1 m1}| sigma_x 4pi Y_l0(z) Y_l0(r) |X_{k2 m2}>   (Eq. Htheta form) */
double or_angular(int kappa1, int two_mu1, int kappa2, int two_mu2, int l)
{
    int l1 = lkap(kappa1), l2 = lkap(kappa2);
    double cu1, cd1, cu2, cd2;
    spinor_cg(kappa1, two_mu1, &cu1, &cd1);
    spinor_cg(kappa2, two_mu2, &cu2, &cd2);
    double res = 0;
    /* sigma_x swaps the spinor rows: conj(X1_up) X2_dn + conj(X1_dn) X2_up */
    int m1 = (two_mu1 - 1) / 2, m2 = (two_mu2 + 1) / 2;
    if (m1 == m2 && abs(m1) <= l1 && abs(m2) <= l2 && cu1 != 0 && cd2 != 0)
        res += cu1 * cd2 * theta_integral(l1, l2, m1, l);
    m1 = (two_mu1 + 1) / 2;
    m2 = (two_mu2 - 1) / 2;
    if (m1 == m2 && abs(m1) <= l1 && abs(m2) <= l2 && cd1 != 0 && cu2 != 0)
        res += cd1 * cu2 * theta_integral(l1, l2, m1, l);
    return res;
}

/* Same coefficient by brute-force 2D quadrature of the spinors on the sphere. */
double or_angular_2d(int kappa1, int two_mu1, int kappa2, int two_mu2, int l, int nth, int nph)
{
    double* x = (double*)malloc(sizeof(double) * nth);
    double* w = (double*)malloc(sizeof(double) * nth);
    or_gauss_legendre(nth, x, w);
    cplx s = 0;
    for (int i = 0; i < nth; i++)
        for (int j = 0; j < nph; j++) {
            double th = acos(x[i]), ph = 2 * M_PI * j / nph;
            double a[4], b[4];
            or_spinor(kappa1, two_mu1, th, ph, a);
            or_spinor(kappa2, two_mu2, th, ph, b);
            cplx a0 = a[0] + I * a[1], a1 = a[2] + I * a[3], b0 = b[0] + I * b[1], b1 = b[2] + I * b[3];
            cplx v = conj(a0) * b1 + conj(a1) * b0;
            s += w[i] * (2 * M_PI / nph) * v * (2 * l + 1) * legendre(l, x[i]);
        }
    free(x); free(w);
    return creal(s);
}

/* ------------------------------------------------------------------------------------------ */
/* Pulse (Eq. ndpPot) and its separable plane-wave form (Eq. bdpA), polarisation x, k along z. */
/* A_x = (E0/w) sin^2(pi s / T) sin(w s), s = t - z / c, switched on for 0 <= t <= T.          */
/* sin(w s) = sin(w t) cos(q z) - cos(w t) sin(q z), q = w / c;                                */
/* cos(qz) = sum_{l even} (-1)^{l/2} (2l+1) j_l(qr) P_l(cos th),                               */
/* sin(qz) = sum_{l odd} (-1)^{(l-1)/2} (2l+1) j_l(qr) P_l(cos th).                             */
/* F_l(t,r) collects everything in front of (2l+1) P_l(cos th).                                */
/* ------------------------------------------------------------------------------------------ */

double or_field_direct(const or_ctx* c, double t, double r, double cos_theta)
{
    if (t < 0 || t > c->T) return 0.0;
    double s = t - r * cos_theta / c->p.c, e = sin(M_PI * s / c->T);
    return c->p.E0 / c->p.omega * e * e * sin(c->p.omega * s);
}

static double time_factor(const or_ctx* c, int cc, int l, double t)
{
    if (l % 2 == 0) return ((l / 2) % 2 ? -1.0 : 1.0) * sin(c->w[cc] * t);
    return -(((l - 1) / 2) % 2 ? -1.0 : 1.0) * cos(c->w[cc] * t);
}

double or_field_F(const or_ctx* c, double t, double r, int l)
{
    if (t < 0 || t > c->T) return 0.0;
    double s = 0;
    for (int cc = 0; cc < 3; cc++) s += c->wt[cc] * time_factor(c, cc, l, t) * or_sph_bessel(l, c->w[cc] * r / c->p.c);
    return c->p.E0 / c->p.omega * s;
}

double or_field_series(const or_ctx* c, double t, double r, double cos_theta, int lmax)
{
    double s = 0;
    for (int l = 0; l <= lmax; l++) s += or_field_F(c, t, r, l) * (2 * l + 1) * legendre(l, cos_theta);
    return s;
}

/* F_l(t, r_p) at every quadrature point, l = 0..l_max: out[l * npts + p] */
static double* field_at_points(const or_ctx* c, double t)
{
    int L = c->p.l_max + 1;
    double* F = (double*)calloc((size_t)L * c->npts, sizeof(double));
    if (t < 0 || t > c->T) return F;
    double amp = c->p.E0 / c->p.omega;
    for (int l = 0; l < L; l++)
        for (int cc = 0; cc < 3; cc++) {
            double f = amp * c->wt[cc] * time_factor(c, cc, l, t);
            const double* j = &c->jl[(cc * L + l) * c->npts];
            for (int pp = 0; pp < c->npts; pp++) F[l * c->npts + pp] += f * j[pp];
        }
    return F;
}

/* ------------------------------------------------------------------------------------------ */
/* Channel adjacency: b is a neighbour of a when some l <= l_max gives a nonzero A1_l or A2_l. */
/* ------------------------------------------------------------------------------------------ */

static void ensure_adj(or_ctx* c, int a)
{
    if (c->adj_done[a]) return;
    int L = c->p.l_max + 1, cnt = 0;
    struct edge_info* list = (struct edge_info*)malloc(sizeof(struct edge_info) * c->nch);
    for (int b = 0; b < c->nch; b++) {
        if (abs(c->tmu[b] - c->tmu[a]) != 2) continue;
        double* A1 = (double*)malloc(sizeof(double) * L);
        double* A2 = (double*)malloc(sizeof(double) * L);
        int nz = 0;
        for (int l = 0; l < L; l++) {
            A1[l] = or_angular(c->kap[a], c->tmu[a], -c->kap[b], c->tmu[b], l);
            A2[l] = or_angular(-c->kap[a], c->tmu[a], c->kap[b], c->tmu[b], l);
            if (fabs(A1[l]) < 1e-13) A1[l] = 0;
            if (fabs(A2[l]) < 1e-13) A2[l] = 0;
            if (A1[l] != 0 || A2[l] != 0) nz = 1;
        }
        if (nz) { list[cnt].b = b; list[cnt].A1 = A1; list[cnt].A2 = A2; cnt++; }
        else { free(A1); free(A2); }
    }
    c->adj[a] = list;
    c->nadj[a] = cnt;
    c->adj_done[a] = 1;
}

static void ensure_all_adj(or_ctx* c)
{
    /* build in parallel: every channel writes only its own slot */
    #pragma omp parallel for schedule(dynamic)
    for (int a = 0; a < c->nch; a++) ensure_adj(c, a);
}

int or_nedges(or_ctx* c)
{
    ensure_all_adj(c);
    int n = 0;
    for (int a = 0; a < c->nch; a++) n += c->nadj[a];
    return n;
}

void or_edges(or_ctx* c, int* ea, int* eb)
{
    ensure_all_adj(c);
    int n = 0;
    for (int a = 0; a < c->nch; a++)
        for (int e = 0; e < c->nadj[a]; e++) { ea[n] = a; eb[n] = c->adj[a][e].b; n++; }
}

/* ------------------------------------------------------------------------------------------ */
/* Interaction H_I = -c alpha.A between psi_{a,i} = (1/r)(P_i X_{ka ma}, i Q_i X_{-ka ma}) and  */
/* psi_{b,j}:  <a i|H_I|b j> = -i c int dr dOmega A_x [ P_i Q_j X_a^+ sigma_x X_{-b}            */
/*                                                   - Q_i P_j X_{-a}^+ sigma_x X_b ]           */
/*                          = i X_ab[i][j],                                                     */
/* X_ab[i][j] = -c sum_l [ A1_l int P_i F_l Q_j dr - A2_l int Q_i F_l P_j dr ].                */
/* ------------------------------------------------------------------------------------------ */

static double coupling_elem(const or_ctx* c, int ka, int kb, const double* A1, const double* A2,
                            int i, int j, const double* F)
{
    int p0, p1;
    if (!common_points(c, i, j, &p0, &p1)) return 0.0;
    int L = c->p.l_max + 1;
    double acc = 0;
    for (int pp = p0; pp < p1; pp++) {
        double Pi, dPi, Qi, dQi, Pj, dPj, Qj, dQj;
        dkb(c, pp, ka, i, &Pi, &dPi, &Qi, &dQi);
        dkb(c, pp, kb, j, &Pj, &dPj, &Qj, &dQj);
        double f1 = 0, f2 = 0;
        for (int l = 0; l < L; l++) {
            f1 += A1[l] * F[l * c->npts + pp];
            f2 += A2[l] * F[l * c->npts + pp];
        }
        acc += c->pw[pp] * (f1 * Pi * Qj - f2 * Qi * Pj);
    }
    return -c->p.c * acc;
}

void or_coupling_block(or_ctx* c, int a, int b, double t, double* X)
{
    int n = dim2(c), L = c->p.l_max + 1;
    double* A1 = (double*)malloc(sizeof(double) * L);
    double* A2 = (double*)malloc(sizeof(double) * L);
    for (int l = 0; l < L; l++) {
        A1[l] = or_angular(c->kap[a], c->tmu[a], -c->kap[b], c->tmu[b], l);
        A2[l] = or_angular(-c->kap[a], c->tmu[a], c->kap[b], c->tmu[b], l);
    }
    double* F = field_at_points(c, t);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) X[(size_t)i * n + j] = coupling_elem(c, c->kap[a], c->kap[b], A1, A2, i, j, F);
    free(F); free(A1); free(A2);
}

void or_coupling_3d(or_ctx* c, int a, int i, int b, int j, double t, int nth, int nph, double* out2)
{
    double* x = (double*)malloc(sizeof(double) * nth);
    double* w = (double*)malloc(sizeof(double) * nth);
    or_gauss_legendre(nth, x, w);
    cplx s = 0;
    int p0, p1;
    if (common_points(c, i, j, &p0, &p1))
        for (int pp = p0; pp < p1; pp++) {
            double Pi, dPi, Qi, dQi, Pj, dPj, Qj, dQj;
            dkb(c, pp, c->kap[a], i, &Pi, &dPi, &Qi, &dQi);
            dkb(c, pp, c->kap[b], j, &Pj, &dPj, &Qj, &dQj);
            double r = c->pr[pp];
            for (int it = 0; it < nth; it++)
                for (int ip = 0; ip < nph; ip++) {
                    double th = acos(x[it]), ph = 2 * M_PI * ip / nph;
                    double Xa[4], Xma[4], Xb[4], Xmb[4];
                    or_spinor(c->kap[a], c->tmu[a], th, ph, Xa);
                    or_spinor(-c->kap[a], c->tmu[a], th, ph, Xma);
                    or_spinor(c->kap[b], c->tmu[b], th, ph, Xb);
                    or_spinor(-c->kap[b], c->tmu[b], th, ph, Xmb);
                    /* four-spinors (without the common 1/r): (P X, i Q X_-) */
                    cplx ua[4] = {Pi * (Xa[0] + I * Xa[1]), Pi * (Xa[2] + I * Xa[3]),
                                  I * Qi * (Xma[0] + I * Xma[1]), I * Qi * (Xma[2] + I * Xma[3])};
                    cplx ub[4] = {Pj * (Xb[0] + I * Xb[1]), Pj * (Xb[2] + I * Xb[3]),
                                  I * Qj * (Xmb[0] + I * Xmb[1]), I * Qj * (Xmb[2] + I * Xmb[3])};
                    /* alpha_x = [[0, sigma_x], [sigma_x, 0]]: rows (0,1,2,3) <- (3,2,1,0) */
                    cplx ax[4] = {ub[3], ub[2], ub[1], ub[0]};
                    cplx dot = 0;
                    for (int q = 0; q < 4; q++) dot += conj(ua[q]) * ax[q];
                    double A = or_field_direct(c, t, r, x[it]);
                    s += c->pw[pp] * w[it] * (2 * M_PI / nph) * (-c->p.c * A) * dot;
                }
        }
    free(x); free(w);
    out2[0] = creal(s);
    out2[1] = cimag(s);
}

/* ------------------------------------------------------------------------------------------ */
/* Operator A_+-(t) = S +- i tau (H0 + i X(t)) = S +- i tau H0 -+ tau X(t),  tau = dt / 2.      */
/* ------------------------------------------------------------------------------------------ */

static void ensure_coupling_cache(or_ctx* c, double t)
{
    if (c->cache_ok && c->cache_t == t) return;
    drop_coupling_cache(c);
    ensure_all_adj(c);
    int n = dim2(c);
    double* F = field_at_points(c, t);
    for (int a = 0; a < c->nch; a++) c->X[a] = (double**)calloc(c->nadj[a] ? c->nadj[a] : 1, sizeof(double*));
    #pragma omp parallel for schedule(dynamic)
    for (int a = 0; a < c->nch; a++)
        for (int e = 0; e < c->nadj[a]; e++) {
            struct edge_info* ed = &c->adj[a][e];
            double* X = (double*)malloc(sizeof(double) * n * n);
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++)
                    X[(size_t)i * n + j] = coupling_elem(c, c->kap[a], c->kap[ed->b], ed->A1, ed->A2, i, j, F);
            c->X[a][e] = X;
        }
    free(F);
    c->cache_t = t;
    c->cache_ok = 1;
}

void or_apply(or_ctx* c, double t, int sign, const double* xd, double* yd)
{
    int n = dim2(c);
    for (int a = 0; a < c->nch; a++) ensure_radial(c, c->kap[a]);
    ensure_coupling_cache(c, t);
    double tau = 0.5 * c->p.dt;
    const cplx* x = (const cplx*)xd;
    cplx* y = (cplx*)yd;
    #pragma omp parallel for schedule(dynamic)
    for (int a = 0; a < c->nch; a++) {
        const double* S = c->S[kslot(c->kap[a])];
        const double* H = c->H[kslot(c->kap[a])];
        const cplx* xa = x + (size_t)a * n;
        cplx* ya = y + (size_t)a * n;
        for (int i = 0; i < n; i++) {
            if (!active(c, c->kap[a], i)) { ya[i] = xa[i]; continue; } /* identity on unused slots */
            cplx acc = 0;
            for (int j = 0; j < n; j++) acc += (S[(size_t)i * n + j] + sign * I * tau * H[(size_t)i * n + j]) * xa[j];
            for (int e = 0; e < c->nadj[a]; e++) {
                const double* X = c->X[a][e];
                const cplx* xb = x + (size_t)c->adj[a][e].b * n;
                for (int j = 0; j < n; j++) acc += -sign * tau * X[(size_t)i * n + j] * xb[j];
            }
            ya[i] = acc;
        }
    }
}

void or_apply_rows(or_ctx* c, double t, int sign, const double* xd, int nrows, const int* ch,
                   const int* idx, double* out)
{
    int n = dim2(c);
    double tau = 0.5 * c->p.dt;
    const cplx* x = (const cplx*)xd;
    double* F = field_at_points(c, t);
    for (int r = 0; r < nrows; r++) ensure_adj(c, ch[r]);
    #pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < nrows; r++) {
        int a = ch[r], i = idx[r];
        const cplx* xa = x + (size_t)a * n;
        cplx acc = 0;
        if (!active(c, c->kap[a], i)) {
            out[2 * r] = creal(xa[i]);
            out[2 * r + 1] = cimag(xa[i]);
            continue;
        }
        for (int j = 0; j < n; j++) {
            double s, h;
            radial_elem(c, c->kap[a], i, j, &s, &h);
            if (s != 0 || h != 0) acc += (s + sign * I * tau * h) * xa[j];
        }
        for (int e = 0; e < c->nadj[a]; e++) {
            struct edge_info* ed = &c->adj[a][e];
            const cplx* xb = x + (size_t)ed->b * n;
            for (int j = 0; j < n; j++) {
                double v = coupling_elem(c, c->kap[a], c->kap[ed->b], ed->A1, ed->A2, i, j, F);
                if (v != 0) acc += -sign * tau * v * xb[j];
            }
        }
        out[2 * r] = creal(acc);
        out[2 * r + 1] = cimag(acc);
    }
    free(F);
}

void or_dense_operator(or_ctx* c, double t, int sign, double* Ad)
{
    int n = dim2(c), nt = n * c->nch;
    cplx* A = (cplx*)Ad;
    memset(A, 0, sizeof(cplx) * (size_t)nt * nt);
    for (int a = 0; a < c->nch; a++) ensure_radial(c, c->kap[a]);
    ensure_coupling_cache(c, t);
    double tau = 0.5 * c->p.dt;
    for (int a = 0; a < c->nch; a++) {
        const double* S = c->S[kslot(c->kap[a])];
        const double* H = c->H[kslot(c->kap[a])];
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                A[(size_t)(a * n + i) * nt + a * n + j] = S[(size_t)i * n + j] + sign * I * tau * H[(size_t)i * n + j];
        for (int i = 0; i < n; i++)
            if (!active(c, c->kap[a], i)) A[(size_t)(a * n + i) * nt + a * n + i] = 1;
        for (int e = 0; e < c->nadj[a]; e++) {
            int b = c->adj[a][e].b;
            const double* X = c->X[a][e];
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++) A[(size_t)(a * n + i) * nt + b * n + j] = -sign * tau * X[(size_t)i * n + j];
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Dense complex LU with partial pivoting                                                      */
/* ------------------------------------------------------------------------------------------ */

static int lu_factor(int n, cplx* A, int* piv)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = cabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; i++)
            if (cabs(A[(size_t)i * n + k]) > best) { best = cabs(A[(size_t)i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0) return -1;
        if (p != k)
            for (int j = 0; j < n; j++) {
                cplx tmp = A[(size_t)k * n + j];
                A[(size_t)k * n + j] = A[(size_t)p * n + j];
                A[(size_t)p * n + j] = tmp;
            }
        for (int i = k + 1; i < n; i++) {
            cplx f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            A[(size_t)i * n + k] = f;
            if (f != 0)
                for (int j = k + 1; j < n; j++) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
        }
    }
    return 0;
}

static void lu_solve(int n, const cplx* LU, const int* piv, cplx* b)
{
    for (int k = 0; k < n; k++)
        if (piv[k] != k) { cplx t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < i; j++) b[i] -= LU[(size_t)i * n + j] * b[j];
    for (int i = n - 1; i >= 0; i--) {
        for (int j = i + 1; j < n; j++) b[i] -= LU[(size_t)i * n + j] * b[j];
        b[i] /= LU[(size_t)i * n + i];
    }
}

int or_dense_solve(int n, const double* Ad, const double* bd, double* xd)
{
    cplx* A = (cplx*)malloc(sizeof(cplx) * (size_t)n * n);
    int* piv = (int*)malloc(sizeof(int) * n);
    memcpy(A, Ad, sizeof(cplx) * (size_t)n * n);
    memcpy(xd, bd, sizeof(cplx) * n);
    int rc = lu_factor(n, A, piv);
    if (rc == 0) lu_solve(n, A, piv, (cplx*)xd);
    free(A); free(piv);
    return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Preconditioner (Eq. matrixM): M = S + i dt/2 H0, block diagonal, one dense LU per kappa.    */
/* ------------------------------------------------------------------------------------------ */

static void ensure_precond(or_ctx* c, int kappa)
{
    int sl = kslot(kappa), n = dim2(c);
    if (c->Mlu[sl]) return;
    ensure_radial(c, kappa);
    double tau = 0.5 * c->p.dt;
    cplx* M = (cplx*)malloc(sizeof(cplx) * (size_t)n * n);
    for (size_t e = 0; e < (size_t)n * n; e++) M[e] = c->S[sl][e] + I * tau * c->H[sl][e];
    for (int i = 0; i < n; i++)
        if (!active(c, kappa, i)) M[(size_t)i * n + i] = 1;
    int* piv = (int*)malloc(sizeof(int) * n);
    lu_factor(n, M, piv);
    c->Mlu[sl] = M;
    c->Mpiv[sl] = piv;
}

void or_precond(or_ctx* c, const double* rd, double* zd)
{
    int n = dim2(c);
    for (int a = 0; a < c->nch; a++) ensure_precond(c, c->kap[a]);
    const cplx* r = (const cplx*)rd;
    cplx* z = (cplx*)zd;
    #pragma omp parallel for
    for (int a = 0; a < c->nch; a++) {
        int sl = kslot(c->kap[a]);
        memcpy(z + (size_t)a * n, r + (size_t)a * n, sizeof(cplx) * n);
        lu_solve(n, c->Mlu[sl], c->Mpiv[sl], z + (size_t)a * n);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* BiCGSTAB (right preconditioned, complex, <u,v> = u^H v), stopped on the true residual      */
/* ||b - A x|| <= tol ||b||; on breakdown or a recursive/true residual mismatch it restarts.   */
/* ------------------------------------------------------------------------------------------ */

static cplx dotc(size_t n, const cplx* u, const cplx* v)
{
    cplx s = 0;
    for (size_t i = 0; i < n; i++) s += conj(u[i]) * v[i];
    return s;
}
static double nrm2(size_t n, const cplx* u) { return sqrt(creal(dotc(n, u, u))); }

static void prec_or_copy(or_ctx* c, int precond, const cplx* in, cplx* out, size_t n)
{
    if (precond) or_precond(c, (const double*)in, (double*)out);
    else memcpy(out, in, sizeof(cplx) * n);
}

int or_step(or_ctx* c, double* psid, double t_n, double tol, int max_iter, int precond, double* resid_out)
{
    size_t n = (size_t)dim2(c) * c->nch;
    double ts = t_n + (c->p.time_eval ? c->p.dt : 0.5 * c->p.dt);
    cplx* psi = (cplx*)psid;
    cplx *b = malloc(sizeof(cplx) * n), *x = malloc(sizeof(cplx) * n), *r = malloc(sizeof(cplx) * n);
    cplx *rh = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n), *v = malloc(sizeof(cplx) * n);
    cplx *ph = malloc(sizeof(cplx) * n), *s = malloc(sizeof(cplx) * n), *sh = malloc(sizeof(cplx) * n);
    cplx *tt = malloc(sizeof(cplx) * n);
    or_apply(c, ts, -1, psid, (double*)b);
    memcpy(x, psi, sizeof(cplx) * n);
    double bn = nrm2(n, b);
    if (bn == 0) bn = 1;
    int it = 0, done = 0;
    double res = 0;
    while (!done && it < max_iter) {
        or_apply(c, ts, +1, (double*)x, (double*)r);
        for (size_t e = 0; e < n; e++) r[e] = b[e] - r[e];
        res = nrm2(n, r) / bn;
        if (res <= tol) break;
        memcpy(rh, r, sizeof(cplx) * n);
        cplx rho_prev = 1, alpha = 1, omega = 1;
        memset(v, 0, sizeof(cplx) * n);
        memset(p, 0, sizeof(cplx) * n);
        while (it < max_iter) {
            it++;
            cplx rho = dotc(n, rh, r);
            if (cabs(rho) == 0) break; /* breakdown: restart from x */
            cplx beta = (rho / rho_prev) * (alpha / omega);
            for (size_t e = 0; e < n; e++) p[e] = r[e] + beta * (p[e] - omega * v[e]);
            prec_or_copy(c, precond, p, ph, n);
            or_apply(c, ts, +1, (double*)ph, (double*)v);
            cplx rv = dotc(n, rh, v);
            if (cabs(rv) == 0) break;
            alpha = rho / rv;
            for (size_t e = 0; e < n; e++) s[e] = r[e] - alpha * v[e];
            if (nrm2(n, s) / bn <= tol) {
                for (size_t e = 0; e < n; e++) x[e] += alpha * ph[e];
                break;
            }
            prec_or_copy(c, precond, s, sh, n);
            or_apply(c, ts, +1, (double*)sh, (double*)tt);
            double tn = creal(dotc(n, tt, tt));
            if (tn == 0) break;
            omega = dotc(n, tt, s) / tn;
            for (size_t e = 0; e < n; e++) x[e] += alpha * ph[e] + omega * sh[e];
            for (size_t e = 0; e < n; e++) r[e] = s[e] - omega * tt[e];
            if (nrm2(n, r) / bn <= tol) break;
            if (cabs(omega) == 0) break;
            rho_prev = rho;
        }
        /* re-check with the true residual at the top of the loop */
        or_apply(c, ts, +1, (double*)x, (double*)r);
        for (size_t e = 0; e < n; e++) r[e] = b[e] - r[e];
        res = nrm2(n, r) / bn;
        if (res <= tol) done = 1;
    }
    memcpy(psi, x, sizeof(cplx) * n);
    if (resid_out) *resid_out = res;
    free(b); free(x); free(r); free(rh); free(p); free(v); free(ph); free(s); free(sh); free(tt);
    return res <= tol ? it : -1;
}

int or_step_dense(or_ctx* c, double* psid, double t_n)
{
    size_t n = (size_t)dim2(c) * c->nch;
    double ts = t_n + (c->p.time_eval ? c->p.dt : 0.5 * c->p.dt);
    double* A = (double*)malloc(sizeof(cplx) * n * n);
    double* b = (double*)malloc(sizeof(cplx) * n);
    or_apply(c, ts, -1, psid, b);
    or_dense_operator(c, ts, +1, A);
    int rc = or_dense_solve((int)n, A, b, psid);
    free(A); free(b);
    return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Generalised symmetric eigenproblem H0 v = E S v (Sec. 2.3): Cholesky S = L L^T, cyclic      */
/* Jacobi on L^-1 H0 L^-T, v = L^-T y.  Eigenvalues ascending; v^T S v = 1; largest-magnitude  */
/* component of each v positive.                                                              */
/* ------------------------------------------------------------------------------------------ */

static void jacobi_eigen(int n, double* A, double* Vv, double* e)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) Vv[(size_t)i * n + j] = i == j;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                double a2 = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += a2;
                if (i != j) off += a2;
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = A[(size_t)p * n + q];
                if (fabs(apq) < 1e-300) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double theta = (aqq - app) / (2 * apq);
                double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1));
                double cs = 1 / sqrt(tt * tt + 1), sn = tt * cs;
                for (int k = 0; k < n; k++) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = cs * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; k++) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = cs * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; k++) {
                    double vkp = Vv[(size_t)k * n + p], vkq = Vv[(size_t)k * n + q];
                    Vv[(size_t)k * n + p] = cs * vkp - sn * vkq;
                    Vv[(size_t)k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
    for (int i = 0; i < n; i++) e[i] = A[(size_t)i * n + i];
}

static void ensure_eigen(or_ctx* c, int kappa)
{
    int sl = kslot(kappa), nb = dim2(c);
    if (c->E[sl]) return;
    ensure_radial(c, kappa);
    /* restrict to the functions used by this kappa */
    int* act = (int*)malloc(sizeof(int) * nb);
    int n = 0;
    for (int i = 0; i < nb; i++)
        if (active(c, kappa, i)) act[n++] = i;
    double* S = (double*)malloc(sizeof(double) * n * n);
    double* H = (double*)malloc(sizeof(double) * n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            S[(size_t)i * n + j] = c->S[sl][(size_t)act[i] * nb + act[j]];
            H[(size_t)i * n + j] = c->H[sl][(size_t)act[i] * nb + act[j]];
        }
    double* L = (double*)calloc((size_t)n * n, sizeof(double));
    for (int j = 0; j < n; j++) {
        double d = S[(size_t)j * n + j];
        for (int k = 0; k < j; k++) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        L[(size_t)j * n + j] = sqrt(d);
        for (int i = j + 1; i < n; i++) {
            double sum = S[(size_t)i * n + j];
            for (int k = 0; k < j; k++) sum -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = sum / L[(size_t)j * n + j];
        }
    }
    /* C = L^-1 H L^-T: W = L^-1 H (forward substitution per column), then C = L^-1 W^T */
    double* W = (double*)malloc(sizeof(double) * n * n);
    double* Cm = (double*)malloc(sizeof(double) * n * n);
    for (int col = 0; col < n; col++)
        for (int i = 0; i < n; i++) {
            double sum = H[(size_t)i * n + col];
            for (int k = 0; k < i; k++) sum -= L[(size_t)i * n + k] * W[(size_t)k * n + col];
            W[(size_t)i * n + col] = sum / L[(size_t)i * n + i];
        }
    for (int col = 0; col < n; col++)
        for (int i = 0; i < n; i++) {
            double sum = W[(size_t)col * n + i];
            for (int k = 0; k < i; k++) sum -= L[(size_t)i * n + k] * Cm[(size_t)k * n + col];
            Cm[(size_t)i * n + col] = sum / L[(size_t)i * n + i];
        }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < i; j++) {
            double avg = 0.5 * (Cm[(size_t)i * n + j] + Cm[(size_t)j * n + i]);
            Cm[(size_t)i * n + j] = Cm[(size_t)j * n + i] = avg;
        }
    double* Y = (double*)malloc(sizeof(double) * n * n);
    double* e = (double*)malloc(sizeof(double) * n);
    jacobi_eigen(n, Cm, Y, e);
    /* v = L^-T y (back substitution) */
    double* Vr = (double*)malloc(sizeof(double) * n * n);
    for (int col = 0; col < n; col++)
        for (int i = n - 1; i >= 0; i--) {
            double sum = Y[(size_t)i * n + col];
            for (int k = i + 1; k < n; k++) sum -= L[(size_t)k * n + i] * Vr[(size_t)k * n + col];
            Vr[(size_t)i * n + col] = sum / L[(size_t)i * n + i];
        }
    /* sort ascending; eigenvectors stored as rows V[e][0..nb), zero on unused functions */
    int* ord = (int*)malloc(sizeof(int) * n);
    for (int i = 0; i < n; i++) ord[i] = i;
    for (int i = 1; i < n; i++) {
        int key = ord[i], j = i - 1;
        while (j >= 0 && e[ord[j]] > e[key]) { ord[j + 1] = ord[j]; j--; }
        ord[j + 1] = key;
    }
    double* Es = (double*)malloc(sizeof(double) * nb);
    double* Vs = (double*)calloc((size_t)nb * nb, sizeof(double));
    for (int r = 0; r < nb; r++) Es[r] = INFINITY;
    for (int r = 0; r < n; r++) {
        int col = ord[r];
        Es[r] = e[col];
        int big = 0;
        for (int i = 0; i < n; i++)
            if (fabs(Vr[(size_t)i * n + col]) > fabs(Vr[(size_t)big * n + col])) big = i;
        double sg = Vr[(size_t)big * n + col] < 0 ? -1.0 : 1.0;
        for (int i = 0; i < n; i++) Vs[(size_t)r * nb + act[i]] = sg * Vr[(size_t)i * n + col];
    }
    c->E[sl] = Es;
    c->V[sl] = Vs;
    free(act); free(S); free(H); free(L); free(W); free(Cm); free(Y); free(e); free(Vr); free(ord);
}

int or_eigen(or_ctx* c, int kappa, double* E, double* V)
{
    int n = dim2(c), na = 0;
    ensure_eigen(c, kappa);
    memcpy(E, c->E[kslot(kappa)], sizeof(double) * n);
    memcpy(V, c->V[kslot(kappa)], sizeof(double) * n * n);
    for (int i = 0; i < n; i++) na += active(c, kappa, i);
    return na;
}

/* ------------------------------------------------------------------------------------------ */
/* Observables: norm psi^H S psi, <H0> = psi^H H0 psi, ground-state population of the 1s1/2,   */
/* mu = +1/2 channel, and the population of all bound states (-c^2 < E < 0) in every channel. */
/* ------------------------------------------------------------------------------------------ */

void or_observables(or_ctx* c, const double* psid, double* out4)
{
    int n = dim2(c);
    const cplx* psi = (const cplx*)psid;
    double nrm = 0, en = 0, pg = 0, pb = 0;
    double c2 = c->p.c * c->p.c;
    int g = find_channel(c, -1, 1);
    for (int a = 0; a < c->nch; a++) {
        int sl = kslot(c->kap[a]);
        ensure_eigen(c, c->kap[a]);
        const double* S = c->S[sl];
        const double* H = c->H[sl];
        const cplx* x = psi + (size_t)a * n;
        cplx* Sx = (cplx*)malloc(sizeof(cplx) * n);
        for (int i = 0; i < n; i++) {
            cplx s = 0, h = 0;
            for (int j = 0; j < n; j++) { s += S[(size_t)i * n + j] * x[j]; h += H[(size_t)i * n + j] * x[j]; }
            Sx[i] = s;
            nrm += creal(conj(x[i]) * s);
            en += creal(conj(x[i]) * h);
        }
        int first_pos = -1;
        for (int e = 0; e < n; e++) {
            double E = c->E[sl][e];
            if (E <= -c2 || E >= 0) continue;
            if (first_pos < 0) first_pos = e;
            cplx pr = 0;
            for (int i = 0; i < n; i++) pr += c->V[sl][(size_t)e * n + i] * Sx[i];
            double p2 = creal(pr * conj(pr));
            pb += p2;
            if (a == g && e == first_pos) pg = p2;
        }
        free(Sx);
    }
    out4[0] = nrm;
    out4[1] = en;
    out4[2] = pg;
    out4[3] = pb;
}
