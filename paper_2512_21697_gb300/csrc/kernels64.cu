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
// Coupling assembly: W_ab = tau X_ab(t) for every coupled pair a < b,
//   W[r][d][t][u] = sum_terms sum_n cA[n] G^n_l[r][d][t][u] + cB[n] G^n_l[r'][2h-d][u][t],
// r' = r + d - h; functions unused at slot 0 give zero rows/columns.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ bool used_fn(int kappa, int slot, int type)
{
    return slot != 0 || (type == 0 ? kappa == -1 : kappa == 1);
}

__global__ void k_assemble64(OpView A, const double* G, double* W)
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
    double2* out = reinterpret_cast<double2*>(W + ((p * A.n1 + r) * A.bd + d) * 4);
    out[0] = make_double2(w00, w01);
    out[1] = make_double2(w10, w11);
    }
}

// ---------------------------------------------------------------------------------------------
// y = A_sign x  with  A_+- = S +- i tau H0  -+ (coupling):  for channel a,
//   y_a = (S + sign i tau H0)_{kappa_a} x_a - sign sum_{b>a} W_ab x_b + sign sum_{b<a} W_ba^T x_b.
// One thread per (channel, radial slot): both DKB types.  Optional epilogues: y <- bsub - y and a
// per-block partial of <dv, y> (and of <y, y>).
// ---------------------------------------------------------------------------------------------
template <int BD>
__global__ void __launch_bounds__(128) k_apply64(OpView A, int sign, const double2* __restrict__ x,
                                                  const double* __restrict__ W, double2* __restrict__ y,
                                                  const double2* __restrict__ bsub, const double2* __restrict__ dv,
                                                  double2* part_dot, double* part_nrm, const KState* skip)
{
    if (skip && skip->done) return;   // uniform over the grid: the solve already converged
    const int bd = BD > 0 ? BD : A.bd;
    const int half = (bd - 1) / 2;
    int ch = blockIdx.y;
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    double2 y0 = make_double2(0, 0), y1 = make_double2(0, 0);
    const int n1 = A.n1;
    bool act = r < n1;
    if (act) {
        const double2* xa = x + (int64_t)ch * 2 * n1;
        int ks = A.ch_kslot[ch];
        const double* Sk = A.S + ((int64_t)ks * n1 + r) * bd * 4;
        const double* Hk = A.H + ((int64_t)ks * n1 + r) * bd * 4;
        double st = sign * A.tau;
#pragma unroll
        for (int d = 0; d < bd; d++) {
            int rr = r + d - half;
            if (rr < 0 || rr >= n1) continue;
            double2 x0 = xa[2 * rr], x1 = xa[2 * rr + 1];
            double s00 = Sk[d * 4], s01 = Sk[d * 4 + 1], s10 = Sk[d * 4 + 2], s11 = Sk[d * 4 + 3];
            double h00 = st * Hk[d * 4], h01 = st * Hk[d * 4 + 1], h10 = st * Hk[d * 4 + 2], h11 = st * Hk[d * 4 + 3];
            y0.x += s00 * x0.x + s01 * x1.x - (h00 * x0.y + h01 * x1.y);
            y0.y += s00 * x0.y + s01 * x1.y + (h00 * x0.x + h01 * x1.x);
            y1.x += s10 * x0.x + s11 * x1.x - (h10 * x0.y + h11 * x1.y);
            y1.y += s10 * x0.y + s11 * x1.y + (h10 * x0.x + h11 * x1.x);
        }
        for (int e = A.adj_start[ch]; e < A.adj_start[ch + 1]; e++) {
            int64_t p = A.adj_pair[e];
            const double2* xb = x + (int64_t)A.adj_nbr[e] * 2 * n1;
            const double* Wp = W + p * n1 * bd * 4;
            if (!A.adj_tr[e]) {
                double cs = -sign;
                const double* Wr = Wp + (int64_t)r * bd * 4;
#pragma unroll
                for (int d = 0; d < bd; d++) {
                    int rr = r + d - half;
                    if (rr < 0 || rr >= n1) continue;
                    double2 x0 = xb[2 * rr], x1 = xb[2 * rr + 1];
                    double2 wa = *reinterpret_cast<const double2*>(Wr + d * 4);
                    double2 wb = *reinterpret_cast<const double2*>(Wr + d * 4 + 2);
                    y0.x += cs * (wa.x * x0.x + wa.y * x1.x);
                    y0.y += cs * (wa.x * x0.y + wa.y * x1.y);
                    y1.x += cs * (wb.x * x0.x + wb.y * x1.x);
                    y1.y += cs * (wb.x * x0.y + wb.y * x1.y);
                }
            } else {
                double cs = sign;
#pragma unroll
                for (int d = 0; d < bd; d++) {
                    int rr = r + d - half;
                    if (rr < 0 || rr >= n1) continue;
                    double2 x0 = xb[2 * rr], x1 = xb[2 * rr + 1];
                    const double* Wt = Wp + ((int64_t)rr * bd + (2 * half - d)) * 4;
                    double2 wa = *reinterpret_cast<const double2*>(Wt);
                    double2 wb = *reinterpret_cast<const double2*>(Wt + 2);
                    // (W^T)[t][u] = W[u][t]
                    y0.x += cs * (wa.x * x0.x + wb.x * x1.x);
                    y0.y += cs * (wa.x * x0.y + wb.x * x1.y);
                    y1.x += cs * (wa.y * x0.x + wb.y * x1.x);
                    y1.y += cs * (wa.y * x0.y + wb.y * x1.y);
                }
            }
        }
        int64_t o = (int64_t)ch * 2 * n1 + 2 * r;
        if (bsub) {
            double2 b0 = bsub[o], b1 = bsub[o + 1];
            y0 = make_double2(b0.x - y0.x, b0.y - y0.y);
            y1 = make_double2(b1.x - y1.x, b1.y - y1.y);
        }
        y[o] = y0;
        y[o + 1] = y1;
    }
    if (part_dot || part_nrm) {
        double2 dsum = make_double2(0, 0);
        double nsum = 0;
        if (act) {
            int64_t o = (int64_t)ch * 2 * n1 + 2 * r;
            if (dv) {
                double2 a = cconjmul(dv[o], y0), b = cconjmul(dv[o + 1], y1);
                dsum = make_double2(a.x + b.x, a.y + b.y);
            }
            nsum = y0.x * y0.x + y0.y * y0.y + y1.x * y1.x + y1.y * y1.y;
        }
        block_reduce_store(dsum, nsum, part_dot, part_nrm, (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
    }
}

void launch_apply64(dim3 grid, cudaStream_t st, const OpView& A, int sign, const double2* x, const double* W,
                    double2* y, const double2* bsub, const double2* dv, double2* pdot, double* pnrm,
                    const KState* skip)
{
    if (A.bd == 13)
        k_apply64<13><<<grid, 128, 0, st>>>(A, sign, x, W, y, bsub, dv, pdot, pnrm, skip);
    else
        k_apply64<0><<<grid, 128, 0, st>>>(A, sign, x, W, y, bsub, dv, pdot, pnrm, skip);
}

// ---------------------------------------------------------------------------------------------
// Preconditioner z = M^-1 r (Eq. matrixM), block diagonal over channels; M depends on kappa only.
// One thread per channel, forward substitution with the recorded row interchanges, then back
// substitution with U.  Optional fused prologue: the vector to solve for is formed on the fly,
//   mode 1: p = r + beta (p - omega v)   (written back to p, then z = M^-1 p)
//   mode 2: s = r - alpha v              (written to s, then z = M^-1 s; partial ||s||^2)
// ---------------------------------------------------------------------------------------------
__global__ void k_precond64(OpView A, int mode, const KState* st, const double2* __restrict__ r,
                            const double2* __restrict__ v, double2* __restrict__ io, double2* __restrict__ z,
                            double* part_nrm)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    double nsum = 0;
    if (idx < A.nch && !(st && st->done)) {
        int ch = A.prec_order[idx];
        int n = 2 * A.n1, kb = A.kb, wu = 2 * kb;
        int ks = A.ch_kslot[ch];
        const double2* U = A.luU + (int64_t)ks * n * (wu + 1);
        const double2* L = A.luL + (int64_t)ks * n * kb;
        const int* P = A.luP + (int64_t)ks * n;
        int64_t o = (int64_t)ch * n;
        double2* zc = z + o;
        if (mode == 0) {
            for (int i = 0; i < n; i++) zc[i] = r[o + i];
        } else if (mode == 1) {
            double2 beta = st->beta, omega = st->omega;
            for (int i = 0; i < n; i++) {
                double2 pv = io[o + i], vv = v[o + i];
                double2 t = cmul(omega, vv);
                double2 q = make_double2(pv.x - t.x, pv.y - t.y);
                q = cmul(beta, q);
                double2 rv = r[o + i];
                double2 pn = make_double2(rv.x + q.x, rv.y + q.y);
                io[o + i] = pn;
                zc[i] = pn;
            }
        } else {
            double2 alpha = st->alpha;
            for (int i = 0; i < n; i++) {
                double2 t = cmul(alpha, v[o + i]);
                double2 rv = r[o + i];
                double2 sv = make_double2(rv.x - t.x, rv.y - t.y);
                io[o + i] = sv;
                zc[i] = sv;
                nsum += sv.x * sv.x + sv.y * sv.y;
            }
        }
        for (int j = 0; j < n; j++) {
            int pj = P[j];
            if (pj != j) { double2 t = zc[j]; zc[j] = zc[pj]; zc[pj] = t; }
            double2 zj = zc[j];
            int lim = min(kb, n - 1 - j);
            for (int i = 1; i <= lim; i++) {
                double2 m = cmul(L[(int64_t)j * kb + i - 1], zj);
                zc[j + i].x -= m.x;
                zc[j + i].y -= m.y;
            }
        }
        for (int i = n - 1; i >= 0; i--) {
            double2 s = zc[i];
            int lim = min(wu, n - 1 - i);
            const double2* Ui = U + (int64_t)i * (wu + 1);
            for (int k = 1; k <= lim; k++) {
                double2 m = cmul(Ui[k], zc[i + k]);
                s.x -= m.x;
                s.y -= m.y;
            }
            zc[i] = cdiv(s, Ui[0]);
        }
    }
    if (part_nrm) block_reduce_store(make_double2(0, 0), nsum, nullptr, part_nrm, blockIdx.x);
}

// ---------------------------------------------------------------------------------------------
// BiCGSTAB updates
// ---------------------------------------------------------------------------------------------
// x += alpha ph + omega sh;  r = s - omega t;  partials <rh, r>, ||r||^2.  When the step ended on
// the s-check (done with only alpha), x += alpha ph and nothing else.
__global__ void k_update_xr64(int64_t n, KState* st, double2* x, double2* r, const double2* ph, const double2* sh,
                              const double2* s, const double2* t, const double2* rh, double2* part_dot,
                              double* part_nrm)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double2 dsum = make_double2(0, 0);
    double nsum = 0;
    if (i < n && st->status == 0) {
        double2 a = cmul(st->alpha, ph[i]);
        if (st->done == 2) {   // converged on s: x += alpha ph
            x[i].x += a.x;
            x[i].y += a.y;
        } else if (!st->done) {
            double2 w = cmul(st->omega, sh[i]);
            x[i].x += a.x + w.x;
            x[i].y += a.y + w.y;
            double2 ot = cmul(st->omega, t[i]);
            double2 rn = make_double2(s[i].x - ot.x, s[i].y - ot.y);
            r[i] = rn;
            dsum = cconjmul(rh[i], rn);
            nsum = rn.x * rn.x + rn.y * rn.y;
        }
    }
    block_reduce_store(dsum, nsum, part_dot, part_nrm, blockIdx.x);
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
//       rho = ||r||^2), resets the per-start counters;  2 = alpha = rho / <rh, v>;
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
    if (what == 1) {
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
