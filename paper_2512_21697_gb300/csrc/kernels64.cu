// kernels64.cu -- double-precision kernels of the Crank-Nicolson step (Eq. solPsi):
// pulse factors, coupling assembly (Eq. fullH), block-banded operator apply A_+- x, the
// block-banded LU preconditioner (Eq. matrixM) and the BiCGSTAB vector updates with their
// deterministic two-stage reductions.
#include <cuda_runtime.h>

#include "device.h"
#include "kernels.h"

namespace dg {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b)
{
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// ---------------------------------------------------------------------------------------------
// Pulse time factors s_{l,c}(t) (the f_alpha of Eq. bdpA) and G^n_l(t) = sum_c s_{l,c} g^n_{l,c}.
// ---------------------------------------------------------------------------------------------
__global__ void k_time_factors(PulseView P, const double* t_eval, double* s)
{
    int i = threadIdx.x;
    if (i >= P.L * 3) return;
    int l = i / 3, c = i % 3;
    double tt = *t_eval - P.t0;
    double v = 0;
    if (tt >= 0 && tt <= P.T) {
        double f;
        if (l % 2 == 0) f = ((l / 2) % 2 ? -1.0 : 1.0) * sin(P.w[c] * tt);
        else f = -(((l - 1) / 2) % 2 ? -1.0 : 1.0) * cos(P.w[c] * tt);
        v = P.amp * P.wt[c] * f;
    }
    s[i] = v;
}

__global__ void k_field_combine(PulseView P, int block_elems, const double* s, double* G)
{
    // G[l][n][e] = sum_c s[l][c] M[l][c][n][e],  e over n1*bd*4
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int ln = blockIdx.y;  // l * 4 + n
    if (e >= block_elems) return;
    int l = ln / 4, n = ln % 4;
    double v = 0;
    for (int c = 0; c < 3; c++) v += s[l * 3 + c] * P.M[(((int64_t)l * 3 + c) * 4 + n) * block_elems + e];
    G[(int64_t)ln * block_elems + e] = v;
}

// ---------------------------------------------------------------------------------------------
// Coupling assembly: W_ab = tau X_ab(t) for every coupled pair a < b (and its FP32 rounding
// when W32 is given),
//   W[r][d][t][u] = sum_terms sum_n cA[n] G^n_l[r][d][t][u] + cB[n] G^n_l[r'][2h-d][u][t],
// r' = r + d - h; functions unused at slot 0 give zero rows/columns.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ bool used_fn(int kappa, int slot, int type)
{
    return slot != 0 || (type == 0 ? kappa == -1 : kappa == 1);
}

__global__ void k_assemble64(OpView A, const double* G, double* W, float* W32)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int nrd = A.n1 * A.bd;
    if (idx >= nrd) return;
    for (int64_t p = blockIdx.y; p < A.npairs; p += gridDim.y) {
    int r = idx / A.bd, d = idx - r * A.bd, rr = r + d - A.half;
    double w00 = 0, w01 = 0, w10 = 0, w11 = 0;
    if (rr >= 0 && rr < A.n1) {
        int64_t nb = (int64_t)nrd * 4;   // elements of one band matrix
        for (int q = A.term_start[p]; q < A.term_start[p + 1]; q++) {
            const double* cf = A.term_coef + (int64_t)q * 8;
            const double* Gl = G + (int64_t)A.term_l[q] * 4 * nb;
            for (int n = 0; n < 4; n++) {
                const double* g = Gl + n * nb + ((int64_t)r * A.bd + d) * 4;
                const double* gt = Gl + n * nb + ((int64_t)rr * A.bd + (2 * A.half - d)) * 4;
                double ca = cf[n], cb = cf[4 + n];
                w00 += ca * g[0] + cb * gt[0];
                w01 += ca * g[1] + cb * gt[2];
                w10 += ca * g[2] + cb * gt[1];
                w11 += ca * g[3] + cb * gt[3];
            }
        }
        int ka = A.ch_kappa[A.pair_a[p]], kb = A.ch_kappa[A.pair_b[p]];
        if (!used_fn(ka, r, 0)) w00 = w01 = 0;
        if (!used_fn(ka, r, 1)) w10 = w11 = 0;
        if (!used_fn(kb, rr, 0)) w00 = w10 = 0;
        if (!used_fn(kb, rr, 1)) w01 = w11 = 0;
    }
    int64_t o = ((p * A.n1 + r) * A.bd + d) * 4;
    double2* out = reinterpret_cast<double2*>(W + o);
    out[0] = make_double2(w00, w01);
    out[1] = make_double2(w10, w11);
    if (W32) *reinterpret_cast<float4*>(W32 + o) = make_float4((float)w00, (float)w01, (float)w10, (float)w11);
    }
}

__global__ void k_set_time(double* t_eval, double t) { *t_eval = t; }

__global__ void k_copy64(int64_t n, const double2* a, double2* b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

__global__ void k_zero64(int64_t n, double2* a)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = make_double2(0, 0);
}

// x = c0 a + c1 b + c2 c (real coefficients), for the extrapolated initial guess
__global__ void k_lincomb64(int64_t n, double c0, const double2* a, double c1, const double2* b, double c2,
                            const double2* c, double2* x)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 v = make_double2(c0 * a[i].x, c0 * a[i].y);
    if (b) { v.x += c1 * b[i].x; v.y += c1 * b[i].y; }
    if (c) { v.x += c2 * c[i].x; v.y += c2 * c[i].y; }
    x[i] = v;
}

// ---------------------------------------------------------------------------------------------
// Finishers: one block sums the partials in a fixed order and advances the scalar recurrence.
// ---------------------------------------------------------------------------------------------
__device__ void block_sum_fixed(int np, const double2* pd, const double* pn, double2* od, double* on)
{
    __shared__ double sx[1024], sy[1024], sn[1024];
    int t = threadIdx.x;
    double ax = 0, ay = 0, an = 0;
    for (int i = t; i < np; i += blockDim.x) {
        if (pd) { ax += pd[i].x; ay += pd[i].y; }
        if (pn) an += pn[i];
    }
    sx[t] = ax; sy[t] = ay; sn[t] = an;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w) { sx[t] += sx[t + w]; sy[t] += sy[t + w]; sn[t] += sn[t + w]; }
        __syncthreads();
    }
    if (t == 0) {
        if (od) *od = make_double2(sx[0], sy[0]);
        if (on) *on = sn[0];
    }
}

__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// what: 0 = ||b||^2 into bnorm2 (new step);  1 = Krylov start from r = b - A x (rh = r, so
//       rho = ||r||^2), resets the per-start counters;  8 = as 1 with bnorm2 = ||r||^2;  2 = alpha = rho / <rh, v>;
//       3 = ||s||^2 check;  6 = omega = <t, s> / <t, t> from pd = sum <s, t>, pn = sum ||t||^2;
//       5 = end of iteration: rho = <rh, r>, ||r||^2, beta.
__global__ void k_finish64(int what, KState* st, int np, const double2* pd, const double* pn, const double2* pd2,
                           const double* pn2, int max_iter)
{
    __shared__ double2 d1;
    __shared__ double n1;
    block_sum_fixed(np, pd, pn, &d1, &n1);
    __syncthreads();
    if (threadIdx.x) return;
    if (what == 0) {
        st->bnorm2 = n1;
        st->it = 0; st->done = 0; st->status = 0;
        return;
    }
    if (what == 8) st->bnorm2 = n1;   // tolerance relative to this start (zero initial guess)
    if (what == 1 || what == 8) {
        st->it = 0; st->status = 0;
        st->rnorm2 = n1;
        st->rho = make_double2(n1, 0);
        st->alpha = st->omega = st->rho_prev = make_double2(1, 0);
        st->beta = make_double2(0, 0);
        st->done = (n1 <= st->tol2 * st->bnorm2) ? 1 : 0;
        if (!isfinite(n1)) { st->status = 6; st->done = 1; }
        return;
    }
    if (st->status) return;
    if (what == 5 && st->done == 2) { st->done = 1; return; }   // the s-check finished the solve
    if (st->done) return;
    if (what == 2) {
        double2 rv = d1;
        if (!finite2(rv)) { st->status = 6; st->done = 1; return; }
        if (rv.x == 0 && rv.y == 0) { st->status = 5; st->done = 1; return; }
        st->alpha = cdiv(st->rho, rv);
    } else if (what == 3) {
        st->snorm2 = n1;
        if (!isfinite(n1)) { st->status = 6; st->done = 1; return; }
        if (n1 <= st->tol2 * st->bnorm2) { st->done = 2; st->rnorm2 = n1; st->it++; }
    } else if (what == 6) {
        double2 ts = make_double2(d1.x, -d1.y);   // <t, s> = conj(<s, t>)
        double tt = n1;
        if (!(tt > 0) || !finite2(ts)) { st->status = tt == 0 ? 5 : 6; st->done = 1; return; }
        st->omega = make_double2(ts.x / tt, ts.y / tt);
    } else if (what == 5) {
        st->it++;
        st->rnorm2 = n1;
        if (!isfinite(n1) || !finite2(d1)) { st->status = 6; st->done = 1; return; }
        st->rho_prev = st->rho;
        st->rho = d1;
        if (n1 <= st->tol2 * st->bnorm2) { st->done = 1; return; }
        if ((st->rho.x == 0 && st->rho.y == 0) || (st->omega.x == 0 && st->omega.y == 0)) {
            st->status = 5; st->done = 1; return;
        }
        st->beta = cmul(cdiv(st->rho, st->rho_prev), cdiv(st->alpha, st->omega));
        if (st->it >= max_iter) { st->status = 4; st->done = 1; }
    }
}

}  // namespace dg
