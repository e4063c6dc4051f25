// setup.cpp -- host-side precomputation of libdirac_gb300 (the paper's offline stage, Sec. 3.1
// item 1): knots and B-splines, kappa-polynomial radial matrices, projected pulse matrices,
// angular coefficients from Clebsch-Gordan x Gaunt coefficients, channel pairs, the block-banded
// LU of the preconditioner and the initial 1s state.  All double precision.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace dg {

// ------------------------------------------------------------------------------------------
// Knots (Sec. 2.2): k-fold end knots at 0 and R; breakpoints linear, or linear up to r_lin and
// geometric beyond with the growth factor that lands exactly on R.
// ------------------------------------------------------------------------------------------
static void build_knots(Basis& B)
{
    const auto& p = B.p;
    int m = B.m;
    B.brk.assign(m + 1, 0.0);
    if (p.grid == 1) {
        double h = p.r_lin / p.n_lin;
        int M = m - p.n_lin;
        double span = p.R - p.r_lin;
        // geometric sum h (g + g^2 + ... + g^M) = span; increasing in g, solve by bisection
        auto total = [&](double g) {
            double s = 0, gp = 1;
            for (int i = 0; i < M; i++) { gp *= g; s += gp; }
            return h * s;
        };
        double lo = 1.0, hi = 1.0 + 1.0 / M;
        while (total(hi) < span) hi = 1.0 + 2.0 * (hi - 1.0);
        for (int it = 0; it < 300 && hi - lo > 0; it++) {
            double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            (total(mid) < span ? lo : hi) = mid;
        }
        double g = 0.5 * (lo + hi);
        for (int i = 0; i <= p.n_lin; i++) B.brk[i] = h * i;
        double gp = 1;
        for (int j = 1; j <= M; j++) {
            gp *= g;
            B.brk[p.n_lin + j] = B.brk[p.n_lin + j - 1] + h * gp;
        }
        B.brk[m] = p.R;
    } else {
        for (int i = 0; i <= m; i++) B.brk[i] = p.R * i / m;
    }
    int k = B.k;
    B.knots.clear();
    for (int i = 0; i < k - 1; i++) B.knots.push_back(0.0);
    for (double b : B.brk) B.knots.push_back(b);
    for (int i = 0; i < k - 1; i++) B.knots.push_back(p.R);
}

// de Boor's triangular scheme: the k B-splines nonzero on knot span [t_j, t_{j+1}) at x, of
// every order 1..k, so that derivatives follow from the lower-order values.
// vals[o][i] = B_{j-o+i, o+1}(x), i = 0..o (order o+1).
static void local_bsplines(const std::vector<double>& t, int k, int j, double x,
                           std::vector<std::vector<double>>& vals)
{
    vals.assign(k, std::vector<double>());
    std::vector<double> left(k + 1), right(k + 1);
    std::vector<double> b(1, 1.0);
    vals[0] = b;
    for (int o = 1; o < k; o++) {
        left[o] = x - t[j + 1 - o];
        right[o] = t[j + o] - x;
        std::vector<double> nb(o + 1, 0.0);
        double saved = 0;
        for (int r = 0; r < o; r++) {
            double term = b[r] / (right[r + 1] + left[o - r]);
            nb[r] = saved + right[r + 1] * term;
            saved = left[o - r] * term;
        }
        nb[o] = saved;
        b = nb;
        vals[o] = b;
    }
}

// value, first and second derivative of the order-k splines B_{j-k+1..j} at x
static void spline_derivs(const std::vector<double>& t, int k, int j, double x, double* u, double* du,
                          double* ddu)
{
    std::vector<std::vector<double>> v;
    local_bsplines(t, k, j, x, v);
    // order o+1 spline index s = j - o + i
    auto low = [&](int o, int s) -> double {   // B_{s, o+1}(x), zero outside the local set
        int i = s - (j - o);
        return (i >= 0 && i <= o) ? v[o][i] : 0.0;
    };
    auto dlow = [&](int o, int s) -> double {  // d/dx B_{s, o+1}
        if (o == 0) return 0.0;
        double a = t[s + o] - t[s], b = t[s + o + 1] - t[s + 1];
        double r = 0;
        if (a > 0) r += low(o - 1, s) / a;
        if (b > 0) r -= low(o - 1, s + 1) / b;
        return o * r;
    };
    int o = k - 1;
    for (int i = 0; i < k; i++) {
        int s = j - o + i;
        u[i] = v[o][i];
        du[i] = dlow(o, s);
        double a = t[s + o] - t[s], b = t[s + o + 1] - t[s + 1];
        double r = 0;
        if (a > 0) r += dlow(o - 1, s) / a;
        if (b > 0) r -= dlow(o - 1, s + 1) / b;
        ddu[i] = o * r;
    }
}

// Gauss-Legendre nodes by Newton's method from Tricomi's initial approximation.
static void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(q, 0);
    w.assign(q, 0);
    for (int i = 1; i <= q; i++) {
        double th = M_PI * (4.0 * i - 1.0) / (4.0 * q + 2.0);
        double z = (1.0 - (q - 1.0) / (8.0 * q * q * q)) * std::cos(th);
        double dp = 1;
        for (int it = 0; it < 50; it++) {
            // P_q and P_{q-1} by the three-term recurrence
            double pm = 1.0, pc = z;
            for (int n = 1; n < q; n++) {
                double pn = ((2.0 * n + 1.0) * z * pc - n * pm) / (n + 1.0);
                pm = pc;
                pc = pn;
            }
            if (q == 1) { pc = z; pm = 1.0; }
            dp = q * (pm - z * pc) / (1.0 - z * z);
            double step = pc / dp;
            z -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        x[q - i] = z;
        w[q - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static void build_quadrature(Basis& B)
{
    std::vector<double> gx, gw;
    gauss_legendre(B.p.quad_pts, gx, gw);
    int k = B.k, q = B.p.quad_pts;
    Quad& Q = B.quad;
    Q.r.clear(); Q.w.clear(); Q.first.clear(); Q.u.clear(); Q.du.clear(); Q.ddu.clear();
    std::vector<double> u(k), du(k), ddu(k);
    for (int iv = 0; iv < B.m; iv++) {
        double a = B.brk[iv], b = B.brk[iv + 1];
        int j = k - 1 + iv;  // knot span [t_j, t_{j+1}) = [a, b)
        for (int g = 0; g < q; g++) {
            double x = 0.5 * (a + b) + 0.5 * (b - a) * gx[g];
            spline_derivs(B.knots, k, j, x, u.data(), du.data(), ddu.data());
            Q.r.push_back(x);
            Q.w.push_back(0.5 * (b - a) * gw[g]);
            Q.first.push_back(j - k + 1);
            for (int i = 0; i < k; i++) {
                Q.u.push_back(u[i]);
                Q.du.push_back(du[i]);
                Q.ddu.push_back(ddu[i]);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Dual kinetic balance components, linear in kappa (Eq. dualkinetic):
//   P = p0 + kappa p1, Q = q0 + kappa q1 (and the same for derivatives).
// large: p0 = u, p1 = 0, q0 = u'/2c, q1 = u/(2c r); small: p0 = u'/2c, p1 = -u/(2c r), q0 = u, q1 = 0.
// ------------------------------------------------------------------------------------------
struct DKB {
    double p0, p1, q0, q1, dp0, dp1, dq0, dq1;
};

static DKB dkb_parts(int type, double u, double du, double ddu, double r, double c)
{
    DKB f{};
    double tc = 2 * c, ur = u / r, dur = du / r - u / (r * r);  // d(u/r)/dr
    if (type == 0) {
        f.p0 = u; f.dp0 = du;
        f.q0 = du / tc; f.dq0 = ddu / tc;
        f.q1 = ur / tc; f.dq1 = dur / tc;
    } else {
        f.p0 = du / tc; f.dp0 = ddu / tc;
        f.p1 = -ur / tc; f.dp1 = -dur / tc;
        f.q0 = u; f.dq0 = du;
    }
    return f;
}

bool slot_used(int kappa, int slot, int type)
{
    if (slot != 0) return true;
    return type == 0 ? kappa == -1 : kappa == 1;
}

int kappa_slot(int kappa) { return 2 * (std::abs(kappa) - 1) + (kappa > 0 ? 1 : 0); }

// h_0..h_3, s_0..s_2: H0(kappa) = sum kappa^n h_n, S(kappa) = sum kappa^n s_n, from
//   S  = int (P_i P_j + Q_i Q_j),
//   H0 = int [P_i U P_j + Q_i (U - 2c^2) Q_j - c P_i (Q_j' - kappa Q_j/r) + c Q_i (P_j' + kappa P_j/r)],
// U = -Z/r, expanded in powers of kappa.
static void radial_polynomials(Basis& B)
{
    int n1 = B.n1, half = B.half, k = B.k;
    for (auto& s : B.s) s.init(n1, half);
    for (auto& h : B.h) h.init(n1, half);
    double c = B.p.c, Z = B.p.Z;
    const Quad& Q = B.quad;
    for (size_t pt = 0; pt < Q.r.size(); pt++) {
        double r = Q.r[pt], w = Q.w[pt], U = -Z / r, V = U - 2 * c * c, cr = c / r;
        for (int a = 0; a < k; a++) {
            int sa = Q.first[pt] + a - 1;   // slot = spline index - 1
            if (sa < 0 || sa >= n1) continue;
            for (int b = 0; b < k; b++) {
                int sb = Q.first[pt] + b - 1;
                if (sb < 0 || sb >= n1) continue;
                int d = sb - sa + half;
                for (int ta = 0; ta < 2; ta++) {
                    DKB i = dkb_parts(ta, Q.u[pt * k + a], Q.du[pt * k + a], Q.ddu[pt * k + a], r, c);
                    for (int tb = 0; tb < 2; tb++) {
                        DKB j = dkb_parts(tb, Q.u[pt * k + b], Q.du[pt * k + b], Q.ddu[pt * k + b], r, c);
                        B.s[0].at(sa, d, ta, tb) += w * (i.p0 * j.p0 + i.q0 * j.q0);
                        B.s[1].at(sa, d, ta, tb) += w * (i.p0 * j.p1 + i.p1 * j.p0 + i.q0 * j.q1 + i.q1 * j.q0);
                        B.s[2].at(sa, d, ta, tb) += w * (i.p1 * j.p1 + i.q1 * j.q1);
                        B.h[0].at(sa, d, ta, tb) +=
                            w * (U * i.p0 * j.p0 + V * i.q0 * j.q0 - c * i.p0 * j.dq0 + c * i.q0 * j.dp0);
                        B.h[1].at(sa, d, ta, tb) +=
                            w * (U * (i.p0 * j.p1 + i.p1 * j.p0) + V * (i.q0 * j.q1 + i.q1 * j.q0) -
                                 c * (i.p0 * j.dq1 + i.p1 * j.dq0) + cr * i.p0 * j.q0 +
                                 c * (i.q0 * j.dp1 + i.q1 * j.dp0) + cr * i.q0 * j.p0);
                        B.h[2].at(sa, d, ta, tb) +=
                            w * (U * i.p1 * j.p1 + V * i.q1 * j.q1 - c * i.p1 * j.dq1 +
                                 cr * (i.p0 * j.q1 + i.p1 * j.q0) + c * i.q1 * j.dp1 +
                                 cr * (i.q0 * j.p1 + i.q1 * j.p0));
                        B.h[3].at(sa, d, ta, tb) += w * cr * (i.p1 * j.q1 + i.q1 * j.p1);
                    }
                }
            }
        }
    }
}

void radial_blocks(const Basis& B, int kappa, Band& S, Band& H)
{
    S.init(B.n1, B.half);
    H.init(B.n1, B.half);
    double kp[4] = {1.0, (double)kappa, (double)kappa * kappa, (double)kappa * kappa * kappa};
    for (size_t e = 0; e < S.v.size(); e++) {
        S.v[e] = B.s[0].v[e] + kp[1] * B.s[1].v[e] + kp[2] * B.s[2].v[e];
        H.v[e] = B.h[0].v[e] + kp[1] * B.h[1].v[e] + kp[2] * B.h[2].v[e] + kp[3] * B.h[3].v[e];
    }
    // functions unused by this kappa: zero rows and columns, identity diagonal in S
    for (int t = 0; t < 2; t++) {
        if (slot_used(kappa, 0, t)) continue;
        for (int d = 0; d < B.bd; d++)
            for (int u = 0; u < 2; u++) {
                S.at(0, d, t, u) = H.at(0, d, t, u) = 0;
                int r = d - B.half;  // row slot r >= 0 whose column 0 is this function
                if (r >= 0 && r < B.n1) {
                    int dd = B.half - r;
                    S.at(r, dd, u, t) = H.at(r, dd, u, t) = 0;
                }
            }
        S.at(0, B.half, t, t) = 1.0;
    }
}

// ------------------------------------------------------------------------------------------
// Angular coefficients: Clebsch-Gordan and Gaunt coefficients from the Racah formula for 3j
// symbols (arguments doubled, so half-integers are exact).
// ------------------------------------------------------------------------------------------
static long double factl(int n)
{
    static std::vector<long double> tab;
    if (tab.empty()) {
        tab.resize(400);
        tab[0] = 1;
        for (int i = 1; i < 400; i++) tab[i] = tab[i - 1] * i;
    }
    return (n < 0 || n >= 400) ? 0.0L : tab[n];
}

// Wigner 3j (j1 j2 j3; m1 m2 m3) with every argument given as twice its value
static double threej2(int j1, int j2, int j3, int m1, int m2, int m3)
{
    if (m1 + m2 + m3 != 0) return 0;
    if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0;
    if ((j1 + m1) % 2 || (j2 + m2) % 2 || (j3 + m3) % 2) return 0;
    if (j3 > j1 + j2 || j3 < std::abs(j1 - j2) || (j1 + j2 + j3) % 2) return 0;
    int a = (j1 + j2 - j3) / 2, b = (j1 - j2 + j3) / 2, c = (-j1 + j2 + j3) / 2, s = (j1 + j2 + j3) / 2;
    long double tri = factl(a) * factl(b) * factl(c) / factl(s + 1);
    long double pre = factl((j1 + m1) / 2) * factl((j1 - m1) / 2) * factl((j2 + m2) / 2) *
                      factl((j2 - m2) / 2) * factl((j3 + m3) / 2) * factl((j3 - m3) / 2);
    int kmin = std::max({0, (j2 - j3 - m1) / 2, (j1 - j3 + m2) / 2});
    int kmax = std::min({a, (j1 - m1) / 2, (j2 + m2) / 2});
    long double sum = 0;
    for (int kk = kmin; kk <= kmax; kk++) {
        long double den = factl(kk) * factl((j3 - j2 + m1) / 2 + kk) * factl((j3 - j1 - m2) / 2 + kk) *
                          factl(a - kk) * factl((j1 - m1) / 2 - kk) * factl((j2 + m2) / 2 - kk);
        sum += ((kk % 2) ? -1.0L : 1.0L) / den;
    }
    int ph = (j1 - j2 - m3) / 2;
    long double v = ((ph % 2 + 2) % 2 ? -1.0L : 1.0L) * std::sqrt(tri * pre) * sum;
    return (double)v;
}

// <j1 m1; j2 m2 | J M>, doubled arguments
static double clebsch2(int j1, int m1, int j2, int m2, int J, int M)
{
    int ph = (j1 - j2 + M) / 2;
    double sg = ((ph % 2 + 2) % 2) ? -1.0 : 1.0;
    return sg * std::sqrt(J + 1.0) * threej2(j1, j2, J, m1, m2, -M);
}

// int Y*_{l1 m1} Y_{l m} Y_{l2 m2} dOmega (Eq. GauntCoef with Y* = (-1)^m Y_{l,-m})
static double gaunt_conj(int l1, int m1, int l, int m, int l2, int m2)
{
    double sg = (std::abs(m1) % 2) ? -1.0 : 1.0;
    return sg * std::sqrt((2 * l1 + 1.0) * (2 * l + 1.0) * (2 * l2 + 1.0) / (4 * M_PI)) *
           threej2(2 * l1, 2 * l, 2 * l2, 0, 0, 0) * threej2(2 * l1, 2 * l, 2 * l2, -2 * m1, 2 * m, 2 * m2);
}

static int orbital_l(int kappa) { return kappa > 0 ? kappa : -kappa - 1; }

}  // namespace dg

// 4 pi Y_l0(z) <X_{k1 m1}| sigma_x Y_l0 |X_{k2 m2}>: X = (C_up Y_{l, mu-1/2}, C_dn Y_{l, mu+1/2})
// with C_up = <l mu-1/2; 1/2 1/2 | j mu>, C_dn = <l mu+1/2; 1/2 -1/2 | j mu>; sigma_x swaps the
// spinor rows (Eq. HthetaExpand with the spin projections paired to their own harmonics).
extern "C" double dirac_angular(int k1, int tm1, int k2, int tm2, int l)
{
    using namespace dg;
    int l1 = orbital_l(k1), l2 = orbital_l(k2);
    int j1 = 2 * std::abs(k1) - 1, j2 = 2 * std::abs(k2) - 1;  // doubled j
    auto cup = [](int ll, int tj, int tm) { return clebsch2(2 * ll, tm - 1, 1, 1, tj, tm); };
    auto cdn = [](int ll, int tj, int tm) { return clebsch2(2 * ll, tm + 1, 1, -1, tj, tm); };
    double pref = std::sqrt(4 * M_PI * (2 * l + 1.0));   // 4 pi Y_l0(z)
    double v = 0;
    // bra up-row times sigma_x-swapped ket (ket down-row moved up)
    int mu1u = (tm1 - 1) / 2, mu2d = (tm2 + 1) / 2;
    if (std::abs(mu1u) <= l1 && std::abs(mu2d) <= l2)
        v += cup(l1, j1, tm1) * cdn(l2, j2, tm2) * gaunt_conj(l1, mu1u, l, 0, l2, mu2d);
    int mu1d = (tm1 + 1) / 2, mu2u = (tm2 - 1) / 2;
    if (std::abs(mu1d) <= l1 && std::abs(mu2u) <= l2)
        v += cdn(l1, j1, tm1) * cup(l2, j2, tm2) * gaunt_conj(l1, mu1d, l, 0, l2, mu2u);
    return pref * v;
}

namespace dg {

static void build_channels_and_pairs(Basis& B)
{
    int km = B.p.kappa_max;
    B.kap.clear();
    B.tmu.clear();
    for (int tm = -(2 * km - 1); tm <= 2 * km - 1; tm += 2) {
        if (B.p.two_mu_max > 0 && std::abs(tm) > B.p.two_mu_max) continue;
        for (int ak = 1; ak <= km; ak++)
            for (int sg = -1; sg <= 1; sg += 2)
                if (2 * ak - 1 >= std::abs(tm)) {
                    B.kap.push_back(sg * ak);
                    B.tmu.push_back(tm);
                }
    }
    B.nch = (int)B.kap.size();
    B.pa.clear(); B.pb.clear(); B.pterm.clear();
    B.pterm_start.assign(1, 0);
    for (int a = 0; a < B.nch; a++)
        for (int b = a + 1; b < B.nch; b++) {
            if (std::abs(B.tmu[a] - B.tmu[b]) != 2) continue;
            std::vector<PairTerm> terms;
            for (int l = 0; l <= B.p.l_max; l++) {
                double A1 = dirac_angular(B.kap[a], B.tmu[a], -B.kap[b], B.tmu[b], l);
                double A2 = dirac_angular(-B.kap[a], B.tmu[a], B.kap[b], B.tmu[b], l);
                if (std::fabs(A1) < 1e-13) A1 = 0;
                if (std::fabs(A2) < 1e-13) A2 = 0;
                if (A1 != 0 || A2 != 0) terms.push_back({l, A1, A2});
            }
            if (terms.empty()) continue;
            B.pa.push_back(a);
            B.pb.push_back(b);
            for (auto& t : terms) B.pterm.push_back(t);
            B.pterm_start.push_back((int)B.pterm.size());
        }
}

// ------------------------------------------------------------------------------------------
// Pulse (Eq. ndpPot, Eq. bdpA): sin^2(pi s/T) sin(w s) = 1/2 sin(w s) - 1/4 sin((w + 2pi/T) s)
// - 1/4 sin((w - 2pi/T) s); sin(w' (t - z/c)) = sin(w' t) cos(q z) - cos(w' t) sin(q z) and the
// plane-wave expansion of cos(qz), sin(qz) in (2l+1) j_l(q r) P_l(cos th).  The radial factor
// j_l(q r) is projected on the DKB functions: g^n = int {p0,p1} j_l {q0,q1} dr.
// ------------------------------------------------------------------------------------------
static double sph_j(int l, double x)
{
    // power series x^l / (2l+1)!! * sum_k (-x^2/2)^k / (k! (2l+3)(2l+5)...(2l+2k+1))
    double lead = 1.0;
    for (int i = 1; i <= l; i++) lead *= x / (2.0 * i + 1.0);
    double term = 1.0, sum = 1.0;
    for (int kk = 1; kk < 500; kk++) {
        term *= -x * x / (2.0 * kk * (2.0 * l + 2.0 * kk + 1.0));
        sum += term;
        if (std::fabs(term) <= 1e-18 * std::fabs(sum)) break;
    }
    return lead * sum;
}

void pulse_matrices(const Basis& B, const dirac_pulse& pulse, PulseData& P)
{
    P.T = pulse.n_cycles * 2 * M_PI / pulse.omega;
    P.amp = pulse.E0 / pulse.omega;
    double Om = 2 * M_PI / P.T;
    P.w[0] = pulse.omega;      P.wt[0] = 0.5;
    P.w[1] = pulse.omega + Om; P.wt[1] = -0.25;
    P.w[2] = pulse.omega - Om; P.wt[2] = -0.25;
    P.L = B.p.l_max + 1;
    P.g.assign((size_t)P.L * 3 * 4, Band());
    for (auto& g : P.g) g.init(B.n1, B.half);
    int k = B.k, n1 = B.n1, half = B.half;
    double c = B.p.c;
    const Quad& Q = B.quad;
    std::vector<double> jl((size_t)P.L * 3);
    for (size_t pt = 0; pt < Q.r.size(); pt++) {
        double r = Q.r[pt], w = Q.w[pt];
        for (int l = 0; l < P.L; l++)
            for (int cc = 0; cc < 3; cc++) jl[l * 3 + cc] = w * sph_j(l, P.w[cc] * r / c);
        for (int a = 0; a < k; a++) {
            int sa = Q.first[pt] + a - 1;
            if (sa < 0 || sa >= n1) continue;
            for (int b = 0; b < k; b++) {
                int sb = Q.first[pt] + b - 1;
                if (sb < 0 || sb >= n1) continue;
                int d = sb - sa + half;
                for (int ta = 0; ta < 2; ta++) {
                    DKB i = dkb_parts(ta, Q.u[pt * k + a], Q.du[pt * k + a], Q.ddu[pt * k + a], r, c);
                    for (int tb = 0; tb < 2; tb++) {
                        DKB j = dkb_parts(tb, Q.u[pt * k + b], Q.du[pt * k + b], Q.ddu[pt * k + b], r, c);
                        double v[4] = {i.p0 * j.q0, i.p1 * j.q0, i.p0 * j.q1, i.p1 * j.q1};
                        for (int l = 0; l < P.L; l++)
                            for (int cc = 0; cc < 3; cc++)
                                for (int n = 0; n < 4; n++)
                                    P.g[(l * 3 + cc) * 4 + n].at(sa, d, ta, tb) += jl[l * 3 + cc] * v[n];
                    }
                }
            }
        }
    }
}

double pulse_time_factor(const PulseData& P, const dirac_pulse& pulse, int l, int c, double t)
{
    double tt = t - pulse.t0;
    if (tt < 0 || tt > P.T) return 0.0;
    double f;
    if (l % 2 == 0) f = ((l / 2) % 2 ? -1.0 : 1.0) * std::sin(P.w[c] * tt);
    else f = -(((l - 1) / 2) % 2 ? -1.0 : 1.0) * std::cos(P.w[c] * tt);
    return P.amp * P.wt[c] * f;
}

// ------------------------------------------------------------------------------------------
// Banded LU with partial pivoting (row interchanges recorded per column, multipliers kept in
// the column where they were formed).
// ------------------------------------------------------------------------------------------
template <class T>
template <class F>
bool BandLU<T>::factor(int n_, int kl_, int ku_, F entry)
{
    n = n_; kl = kl_; ku = ku_;
    int wu = kl + ku;                      // fill-in widens U to kl + ku superdiagonals
    int W = kl + wu + 1;                   // working row window [i - kl, i + wu]
    std::vector<T> A((size_t)n * W, T(0));
    auto el = [&](int i, int j) -> T& { return A[(size_t)i * W + (j - i + kl)]; };
    for (int i = 0; i < n; i++)
        for (int j = std::max(0, i - kl); j <= std::min(n - 1, i + ku); j++) el(i, j) = entry(i, j);
    piv.assign(n, 0);
    L.assign((size_t)n * kl, T(0));
    U.assign((size_t)n * (wu + 1), T(0));
    for (int j = 0; j < n; j++) {
        int last = std::min(n - 1, j + kl), p = j;
        double best = std::abs(el(j, j));
        for (int i = j + 1; i <= last; i++)
            if (std::abs(el(i, j)) > best) { best = std::abs(el(i, j)); p = i; }
        if (best == 0) return false;
        piv[j] = p;
        int cend = std::min(n - 1, j + wu);
        if (p != j)
            for (int cc = j; cc <= cend; cc++) std::swap(el(j, cc), el(p, cc));
        T dinv = T(1) / el(j, j);
        for (int i = j + 1; i <= last; i++) {
            T f = el(i, j) * dinv;
            L[(size_t)j * kl + (i - j - 1)] = f;
            if (f != T(0))
                for (int cc = j + 1; cc <= cend; cc++) el(i, cc) -= f * el(j, cc);
        }
        for (int cc = j; cc <= cend; cc++) U[(size_t)j * (wu + 1) + (cc - j)] = el(j, cc);
    }
    return true;
}

template <class T>
void BandLU<T>::solve(T* b) const
{
    int wu = kl + ku;
    for (int j = 0; j < n; j++) {
        if (piv[j] != j) std::swap(b[j], b[piv[j]]);
        for (int i = 1; i <= kl && j + i < n; i++) b[j + i] -= L[(size_t)j * kl + i - 1] * b[j];
    }
    for (int i = n - 1; i >= 0; i--) {
        T s = b[i];
        for (int kk = 1; kk <= wu && i + kk < n; kk++) s -= U[(size_t)i * (wu + 1) + kk] * b[i + kk];
        b[i] = s / U[(size_t)i * (wu + 1)];
    }
}

template struct BandLU<cd>;
template struct BandLU<double>;

// scalar index i = 2 slot + type; entry of a Band as a scalar matrix
double band_entry(const Band& M, int i, int j)
{
    int r = i / 2, t = i % 2, rr = j / 2, u = j % 2;
    int d = rr - r + M.half;
    if (d < 0 || d >= M.bd) return 0.0;
    return M.at(r, d, t, u);
}

bool precond_factor(const Basis& B, int kappa, double tau, BandLU<cd>& lu)
{
    Band S, H;
    radial_blocks(B, kappa, S, H);
    int n = 2 * B.n1, kb = 2 * B.half + 1;
    return lu.factor(n, kb, kb, [&](int i, int j) { return cd(band_entry(S, i, j), tau * band_entry(H, i, j)); });
}

// Initial state (Sec. 2.3): Rayleigh-quotient inverse iteration for the kappa = -1 level
// closest to -Z^2/2 (the 1s1/2 level), H0 v = E S v.
static bool ground_state(Basis& B)
{
    Band S, H;
    radial_blocks(B, -1, S, H);
    int n = 2 * B.n1, kb = 2 * B.half + 1;
    auto Sx = [&](const std::vector<double>& x, std::vector<double>& y, const Band& M) {
        y.assign(n, 0);
        for (int i = 0; i < n; i++)
            for (int j = std::max(0, i - kb); j <= std::min(n - 1, i + kb); j++) y[i] += band_entry(M, i, j) * x[j];
    };
    std::vector<double> v(n, 0.0), y, Sv, Hv;
    for (int i = 0; i < n; i += 2) v[i] = 1.0;  // large components
    v[1] = 0;
    double sigma = -0.5 * B.p.Z * B.p.Z;
    double E = sigma;
    for (int it = 0; it < 60; it++) {
        BandLU<double> lu;
        if (!lu.factor(n, kb, kb, [&](int i, int j) { return band_entry(H, i, j) - sigma * band_entry(S, i, j); }))
            sigma *= 1 + 1e-12;
        Sx(v, Sv, S);
        y = Sv;
        lu.solve(y.data());
        for (int i = 0; i < n; i++)
            if (!slot_used(-1, i / 2, i % 2)) y[i] = 0;
        Sx(y, Sv, S);
        Sx(y, Hv, H);
        double ySy = 0, yHy = 0;
        for (int i = 0; i < n; i++) { ySy += y[i] * Sv[i]; yHy += y[i] * Hv[i]; }
        double nrm = std::sqrt(ySy);
        for (int i = 0; i < n; i++) v[i] = y[i] / nrm;
        double Enew = yHy / ySy;
        bool done = std::fabs(Enew - E) <= 1e-15 * std::fabs(Enew) && it > 3;
        E = Enew;
        if (it >= 2) sigma = E;   // Rayleigh-quotient shift once the direction has settled
        if (done) break;
    }
    int big = 0;
    for (int i = 0; i < n; i++)
        if (std::fabs(v[i]) > std::fabs(v[big])) big = i;
    if (v[big] < 0)
        for (auto& x : v) x = -x;
    B.psi0.assign((size_t)B.n() * 2, 0.0);
    int a = -1;
    for (int ch = 0; ch < B.nch; ch++)
        if (B.kap[ch] == -1 && B.tmu[ch] == 1) a = ch;
    if (a < 0) return false;
    for (int i = 0; i < n; i++) B.psi0[((size_t)a * n + i) * 2] = v[i];
    B.e0 = E;
    return std::isfinite(E);
}

}  // namespace dg

// ------------------------------------------------------------------------------------------
// C ABI: basis
// ------------------------------------------------------------------------------------------
extern "C" dirac_status dirac_basis_build(const dirac_basis_params* p, dirac_basis** out, double* psi0_host,
                                          double* e0)
{
    using namespace dg;
    if (!p || !out) { set_error("dirac_basis_build: NULL argument"); return DIRAC_E_ARG; }
    if (p->order < 3 || p->order > 12 || p->n_splines < p->order || p->kappa_max < 1 || p->kappa_max > 60 ||
        p->l_max < 0 || p->l_max > 40 || p->quad_pts < 1 || p->quad_pts > 64 || !(p->R > 0) || !(p->c > 0) ||
        !(p->Z >= 0)) {
        set_error("dirac_basis_build: parameter out of range");
        return DIRAC_E_ARG;
    }
    int m = p->n_splines + 5 - p->order;
    if (p->grid == 1 && !(p->n_lin > 0 && p->n_lin < m && p->r_lin > 0 && p->r_lin < p->R &&
                          p->R - p->r_lin > (m - p->n_lin) * p->r_lin / p->n_lin)) {
        set_error("dirac_basis_build: grid 1 needs 0 < n_lin < intervals, 0 < r_lin < R and growing intervals");
        return DIRAC_E_ARG;
    }
    if (p->grid != 0 && p->grid != 1) { set_error("dirac_basis_build: grid must be 0 or 1"); return DIRAC_E_ARG; }
    dirac_basis* bas = nullptr;
    try {
        bas = new dirac_basis();
        Basis& B = bas->b;
        B.p = *p;
        B.k = p->order;
        B.half = B.k - 1;
        B.bd = 2 * B.half + 1;
        B.n1 = p->n_splines + 1;
        B.nsp = p->n_splines + 4;
        B.m = m;
        build_knots(B);
        build_quadrature(B);
        radial_polynomials(B);
        build_channels_and_pairs(B);
        if (!ground_state(B)) {
            delete bas;
            set_error("dirac_basis_build: initial state iteration failed (needs kappa = -1, mu = +1/2)");
            return DIRAC_E_NUMERIC;
        }
        if (psi0_host) std::memcpy(psi0_host, B.psi0.data(), sizeof(double) * B.psi0.size());
        if (e0) *e0 = B.e0;
    } catch (const std::bad_alloc&) {
        delete bas;
        set_error("dirac_basis_build: out of host memory");
        return DIRAC_E_NOMEM;
    }
    *out = bas;
    return DIRAC_OK;
}

extern "C" void dirac_basis_free(dirac_basis* b) { delete b; }

extern "C" int64_t dirac_basis_dim(const dirac_basis* b) { return b ? b->b.n() : -1; }

extern "C" int dirac_basis_nchannels(const dirac_basis* b) { return b ? b->b.nch : -1; }

extern "C" int64_t dirac_basis_npairs(const dirac_basis* b) { return b ? (int64_t)b->b.pa.size() : -1; }
extern "C" int64_t dirac_basis_nterms(const dirac_basis* b) { return b ? (int64_t)b->b.pterm.size() : -1; }

extern "C" dirac_status dirac_basis_channels(const dirac_basis* b, int* kappa, int* two_mu)
{
    if (!b || !kappa || !two_mu) { dg::set_error("dirac_basis_channels: NULL argument"); return DIRAC_E_ARG; }
    std::memcpy(kappa, b->b.kap.data(), sizeof(int) * b->b.nch);
    std::memcpy(two_mu, b->b.tmu.data(), sizeof(int) * b->b.nch);
    return DIRAC_OK;
}

extern "C" dirac_status dirac_basis_radial(const dirac_basis* b, int kappa, double* S, double* H0)
{
    using namespace dg;
    if (!b || !S || !H0 || kappa == 0 || std::abs(kappa) > b->b.p.kappa_max) {
        set_error("dirac_basis_radial: bad argument");
        return DIRAC_E_ARG;
    }
    Band Sb, Hb;
    radial_blocks(b->b, kappa, Sb, Hb);
    int n = 2 * b->b.n1;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            S[(size_t)i * n + j] = band_entry(Sb, i, j);
            H0[(size_t)i * n + j] = band_entry(Hb, i, j);
        }
    return DIRAC_OK;
}

extern "C" dirac_status dirac_basis_coupling(const dirac_basis* bas, const dirac_pulse* pulse, int a, int b,
                                             double t, double* X)
{
    using namespace dg;
    if (!bas || !pulse || !X || a < 0 || b < 0 || a >= bas->b.nch || b >= bas->b.nch || a == b) {
        set_error("dirac_basis_coupling: bad argument");
        return DIRAC_E_ARG;
    }
    const Basis& B = bas->b;
    PulseData P;
    pulse_matrices(B, *pulse, P);
    int n = 2 * B.n1;
    std::memset(X, 0, sizeof(double) * n * n);
    double ka = B.kap[a], kb = B.kap[b];
    // X_ab = -c sum_l [A1 int P^{ka} F_l Q^{kb} - A2 (int P^{kb} F_l Q^{ka})^T]
    for (int l = 0; l <= B.p.l_max; l++) {
        double A1 = dirac_angular(B.kap[a], B.tmu[a], -B.kap[b], B.tmu[b], l);
        double A2 = dirac_angular(-B.kap[a], B.tmu[a], B.kap[b], B.tmu[b], l);
        if (A1 == 0 && A2 == 0) continue;
        double mono_ab[4] = {1, ka, kb, ka * kb}, mono_ba[4] = {1, kb, ka, ka * kb};
        for (int cc = 0; cc < 3; cc++) {
            double f = pulse_time_factor(P, *pulse, l, cc, t);
            if (f == 0) continue;
            for (int nn = 0; nn < 4; nn++) {
                const Band& g = P.g[(l * 3 + cc) * 4 + nn];
                for (int i = 0; i < n; i++)
                    for (int j = std::max(0, i - 2 * B.half - 1); j <= std::min(n - 1, i + 2 * B.half + 1); j++) {
                        double v = -B.p.c * f * (A1 * mono_ab[nn] * band_entry(g, i, j) - A2 * mono_ba[nn] * band_entry(g, j, i));
                        X[(size_t)i * n + j] += v;
                    }
            }
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            if (!slot_used(B.kap[a], i / 2, i % 2) || !slot_used(B.kap[b], j / 2, j % 2)) X[(size_t)i * n + j] = 0;
    return DIRAC_OK;
}
