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
// when W32 is given).  With G^n_l = sum_c s_{l,c}(t) g^n_{l,c} and the kappa monomials
// m(k', k) = (1, k', k, k' k), Eq. fullH gives
//   tau X_ab = sum_terms [ -c tau A1 K_l(ka, kb) + c tau A2 K_l(kb, ka)^T ],
//   K_l(k', k) = sum_n m_n(k', k) G^n_l,
// so K is built once per distinct (k', k, l) and shared by every pair (all mu) that uses it.
// Functions unused at slot 0 give zero rows/columns.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ bool used_fn(int kappa, int slot, int type)
{
    return slot != 0 || (type == 0 ? kappa == -1 : kappa == 1);
}

// K[key][e] = sum_n m_n(key) G^n_l[e]  (l = key_l[key]), e over one band
__global__ void k_build_K(OpView A, int block_elems, const double* G, double* K)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= block_elems) return;
    for (int key = blockIdx.y; key < A.nkeys; key += gridDim.y) {
        const double* m = A.key_mono + (int64_t)key * 4;
        const double* Gl = G + (int64_t)A.key_l[key] * 4 * block_elems + e;
        double v = m[0] * Gl[0];
        v = fma(m[1], Gl[block_elems], v);
        v = fma(m[2], Gl[2 * (int64_t)block_elems], v);
        v = fma(m[3], Gl[3 * (int64_t)block_elems], v);
        K[(int64_t)key * block_elems + e] = v;
    }
}

// W_ab[r][d] = sum_terms cA K_l(ka,kb)[r][d] + cB K_l(kb,ka)[r'][2h-d]^T,  r' = r + d - h
__global__ void k_assemble64(OpView A, const double* K, double* W, float* W32)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int nrd = A.n1 * A.bd;
    if (idx >= nrd) return;
    int r = idx / A.bd, d = idx - r * A.bd, rr = r + d - A.half;
    int64_t nb = (int64_t)nrd * 4;   // elements of one band matrix
    for (int64_t pi = blockIdx.y; pi < A.npairs; pi += gridDim.y) {
        int64_t p = A.pair_order[pi];
        double w00 = 0, w01 = 0, w10 = 0, w11 = 0;
        if (rr >= 0 && rr < A.n1) {
            for (int q = A.term_start[p]; q < A.term_start[p + 1]; q++) {
                double ca = A.term_cab[2 * q], cb = A.term_cab[2 * q + 1];
                const double2* g = reinterpret_cast<const double2*>(K + A.term_kd[q] * nb + ((int64_t)r * A.bd + d) * 4);
                const double2* gt =
                    reinterpret_cast<const double2*>(K + A.term_kt[q] * nb + ((int64_t)rr * A.bd + (2 * A.half - d)) * 4);
                double2 g0 = g[0], g1 = g[1], h0 = gt[0], h1 = gt[1];
                w00 = fma(ca, g0.x, fma(cb, h0.x, w00));
                w01 = fma(ca, g0.y, fma(cb, h1.x, w01));
                w10 = fma(ca, g1.x, fma(cb, h0.y, w10));
                w11 = fma(ca, g1.y, fma(cb, h1.y, w11));
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

__global__ void k_set_step_time(double* t_eval, double t_start, int step, double dt, double t_off)
{
    *t_eval = step_time(t_start, step, dt, t_off);
}

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
__global__ void k_extrapolate(int64_t n, int nh, const double2* psi, const double2* h1, const double2* h2, double2* x)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 p = psi[i], a = nh >= 1 ? h1[i] : p, b = nh >= 2 ? h2[i] : p;
    x[i] = make_double2(extrapolate(nh, p.x, a.x, b.x), extrapolate(nh, p.y, a.y, b.y));
}

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
// ||b||^2 of a step's first refinement pass (flag set): bnorm2 = sum of the partials, flag cleared
__global__ void k_bnorm_if(KState* st, int* flag, int np, const double* pn)
{
    __shared__ double2 d1;
    __shared__ double n1;
    if (!*flag) return;   // uniform over the block
    block_sum_fixed(np, nullptr, pn, &d1, &n1);
    __syncthreads();
    if (threadIdx.x) return;
    st->bnorm2 = n1;
    *flag = 0;
}

__global__ void k_set_int(int* p, int v) { *p = v; }

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
