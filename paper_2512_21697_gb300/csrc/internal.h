// internal.h -- host-side data of libdirac_gb300 (basis, operator setup) shared by the
// setup code and the CUDA entry points.  Not part of the public ABI.
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dirac.h"

namespace dg {

using cd = std::complex<double>;

void set_error(const std::string& msg);

// 2x2-block-banded layout: row slot r, block diagonal d (column slot r + d - half), entries
// [row type][column type].  half = order - 1, bd = 2 half + 1.
struct Band {
    int n1 = 0, bd = 0, half = 0;
    std::vector<double> v;  // n1 * bd * 4
    void init(int n1_, int half_) {
        n1 = n1_; half = half_; bd = 2 * half + 1;
        v.assign((size_t)n1 * bd * 4, 0.0);
    }
    double& at(int r, int d, int t, int u) { return v[(((size_t)r * bd + d) * 2 + t) * 2 + u]; }
    double at(int r, int d, int t, int u) const { return v[(((size_t)r * bd + d) * 2 + t) * 2 + u]; }
};

struct Quad {            // Gauss-Legendre points over all knot intervals
    std::vector<double> r, w;
    std::vector<int> first;   // first nonzero B-spline (full-knot-vector index) at the point
    std::vector<double> u, du, ddu;  // [point][order]
};

struct PairTerm {        // one multipole of one coupled channel pair
    int l;
    double A1, A2;       // <X_{ka}|..|X_{-kb}>, <X_{-ka}|..|X_{kb}> (Eq. Htheta coefficients)
};

struct Basis {
    dirac_basis_params p{};
    int k = 0, half = 0, bd = 0, n1 = 0, m = 0, nsp = 0;
    std::vector<double> knots, brk;
    Quad quad;
    int nch = 0;
    std::vector<int> kap, tmu;      // channel labels, library order
    Band s[3], h[4];                // S(kappa) = sum kappa^n s_n, H0(kappa) = sum kappa^n h_n
    std::vector<int> pa, pb;        // coupled pairs a < b
    std::vector<int> pterm_start;   // npairs + 1
    std::vector<PairTerm> pterm;
    std::vector<double> psi0;       // 1s1/2 mu=+1/2 state, library order
    double e0 = 0;
    int64_t n() const { return (int64_t)nch * 2 * n1; }
};

bool slot_used(int kappa, int slot, int type);
int kappa_slot(int kappa);   // 0..2 kappa_max-1

// Radial blocks of one kappa: S, H0 as bands, unused functions replaced by the identity in S
// and zero in H0.
void radial_blocks(const Basis& B, int kappa, Band& S, Band& H);
// scalar entry (i, j) of a Band, i = 2 slot + type (zero outside the band)
double band_entry(const Band& M, int i, int j);

// Pulse: the three carriers of the sin^2 envelope and the projected multipole matrices
// g[l][carrier][n] (Band), n = 0..3 the kappa-polynomial component of int P_i g Q_j dr.
struct PulseData {
    double T = 0, amp = 0;
    double w[3] = {0, 0, 0}, wt[3] = {0, 0, 0};
    int L = 0;
    std::vector<Band> g;   // index (l * 3 + c) * 4 + n
};
void pulse_matrices(const Basis& B, const dirac_pulse& pulse, PulseData& out);
// scalar factor s_{l,c}(t) multiplying g[l][c] (time functions f_alpha of Eq. bdpA)
double pulse_time_factor(const PulseData& P, const dirac_pulse& pulse, int l, int c, double t);

// Banded LU with partial pivoting of an n x n matrix stored as 2x2-block bands (n = 2 n1),
// scalar lower/upper bandwidth kl = ku = 2 half + 1.  U has kl+ku superdiagonals.
template <class T>
struct BandLU {
    int n = 0, kl = 0, ku = 0;
    std::vector<T> L;     // n * kl   multipliers of column j for rows j+1..j+kl
    std::vector<T> U;     // n * (kl+ku+1)  U[i][0] diagonal, U[i][k] column i+k
    std::vector<int> piv;
    // entry(i, j) returns A_ij for |i - j| within the band (zero outside)
    template <class F>
    bool factor(int n_, int kl_, int ku_, F entry);
    void solve(T* b) const;
};

// Assemble the complex matrix M = S + i tau H0 of one kappa as banded LU.
bool precond_factor(const Basis& B, int kappa, double tau, BandLU<cd>& lu);

}  // namespace dg

struct dirac_basis {
    dg::Basis b;
};
