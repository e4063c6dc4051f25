// device.h -- device-side data structures and kernel launchers of libdirac_gb300.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace dg {

// BiCGSTAB scalars (always double precision, Sec. 2.4 / right-preconditioned van der Vorst form).
struct KState {
    double2 rho, rho_prev, alpha, omega, beta;
    double bnorm2, rnorm2, snorm2, tol2;
    int it, done, status, first;
};

// Geometry and operator data read by the kernels.
struct OpView {
    int n1, bd, half, nch;
    int64_t npairs;
    double tau, c;
    const int* ch_kslot;      // [nch] radial-block index of each channel
    const int* ch_kappa;      // [nch]
    const double* S;          // [2 kappa_max][n1][bd][4]
    const double* H;          // [2 kappa_max][n1][bd][4]
    const int* adj_start;     // [nch + 1]
    const int* adj_pair;      // pair of each adjacency entry
    const int* adj_nbr;       // neighbour channel
    const int* adj_tr;        // 0: channel is the pair's lower channel (W x), 1: upper (W^T x)
    const int* own_start;     // [nch + 1] pairs a channel owns (is the lower channel of), in order
    const int* own_pair;
    const int* own_nbr;       // the pair's upper channel
    const int* in_start;      // [nch + 1] pairs a channel is the upper channel of
    const int* in_pair;
    const int* pair_a;        // [npairs]
    const int* pair_b;
    const int* term_start;    // [npairs + 1]
    const int* term_l;        // [nterms]
    const double* term_coef;  // [nterms][8]: cA[4] (direct), cB[4] (transposed), tau included
    // combined radial bands K_l(k', k) = sum_n m_n(k', k) G^n_l, one per distinct (k', k, l)
    int nkeys;
    const int* key_l;         // [nkeys]
    const double* key_mono;   // [nkeys][4]: 1, k', k, k' k
    const int* term_kd;       // [nterms] key of K_l(k_a, k_b)   (direct use)
    const int* term_kt;       // [nterms] key of K_l(k_b, k_a)   (transposed use)
    const double* term_cab;   // [nterms][2]: -c tau A1, c tau A2
    const int* pair_order;    // pairs grouped by (k_a, k_b) so a group's K bands stay in L2
    // preconditioner: per radial block LU of M = S + i tau H0 (scalar bandwidth kb)
    int kb;
    const double2* luU;       // [2 kappa_max][2 n1][2 kb + 1], column form Ucol[i][k] = U[i-k][k]
    const double2* luL;       // [2 kappa_max][2 n1][kb]
    const int* luP;           // [2 kappa_max][2 n1]
    const int* prec_order;    // channels sorted by radial block
    // bounds checking (debug builds, -DDG_BOUNDS): the allocated sizes the checks compare with and
    // a word collecting one bit per kind of violation (null: no checking)
    unsigned int* bounds_err;
    int64_t nb_part;          // owner/gather partial slots as allocated (one float4 each)
    int64_t nb_coup;          // stored coupling values per buffer (floats or doubles)
};

// DG_INB(A, cond, bit): true if cond holds; in a debug build a failed check also records bit in the
// op's bounds word, and the caller skips (or redirects) the access.  Release builds: always true.
#ifdef DG_BOUNDS
__device__ __forceinline__ bool dg_inb(const OpView& A, bool ok, int bit)
{
    if (!ok && A.bounds_err) atomicOr(A.bounds_err, 1u << bit);
    return ok;
}
#define DG_INB(A, cond, bit) dg_inb((A), (cond), (bit))
#else
#define DG_INB(A, cond, bit) true
#endif

// One chunk of a (kappa_a, kappa_b) pair group for the grouped double-float assembly: pairs
// first .. first + count - 1 of the group-ordered pair list and the group's nl multipoles
// (increasing l).
constexpr int ASM_MAX_NL = 4;
constexpr int ASM_CHUNK = 64;
struct AsmChunk {
    int first, count, nl, ka, kb;
    int l[ASM_MAX_NL];
};

// Factorised complex64 apply: radial tiles of FTR rows; the band products of up to FCOL channels
// of one kappa (consecutive in the kappa-sorted channel order, from index first) per block.
constexpr int FTR = 64;
constexpr int FCOL = 8;
struct RadChunk {
    int ks, kappa, first, count;
};
// The subgroup form of the factorised apply: the radial pass puts up to FLANE channels of one kappa
// on the lanes of a warp (their band entries are the same); the angular pass gives a block FSG
// output channels of one mu.  Every partner of a channel has mu +- 1, so the outputs of one mu share
// their partners' band products: an "item" is one (partner, multipole) product set, loaded once per
// block and applied to all FSG outputs with one float4 of coefficients per output (zero where the
// output does not use it).
constexpr int FLANE = 32;
constexpr int FSG = 8;
struct RadPack {          // one radial block: up to two kappa chunks, c[0].count + c[1].count <= FLANE lanes
    RadChunk c[2];
};
struct FactSub {
    int first, count;     // items first .. first + count - 1 of the item lists
    int out[FSG];         // output channels (-1: slot unused)
};

struct PulseView {
    int L;
    double T, amp, t0, dt;
    double w[3], wt[3];
    const double* M;          // [L][3][4][n1][bd][4]
};

}  // namespace dg
