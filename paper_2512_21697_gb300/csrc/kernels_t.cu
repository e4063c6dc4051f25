// kernels_t.cu -- the Krylov-loop kernels in both working precisions (T = double or float):
// block-banded operator apply A_+- x (Eq. solPsi with the coupling of Eq. fullH), the
// block-banded LU preconditioner (Eq. matrixM) with fused BiCGSTAB prologues, and the
// BiCGSTAB solution/residual update.  Per-thread arithmetic is in T; every reduction is summed in
// double and the BiCGSTAB scalars (rho, alpha, omega, beta) are double (KState).
#include <cuda_runtime.h>

#include "device.h"
#include "kernels.h"

namespace dg {

template <class T> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };
template <class T> using c2 = typename C2<T>::t;

template <class T> __device__ __forceinline__ c2<T> mk(T a, T b) { c2<T> v; v.x = a; v.y = b; return v; }
template <class T> __device__ __forceinline__ c2<T> cm(c2<T> a, c2<T> b) { return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <class T> __device__ __forceinline__ c2<T> cdv(c2<T> a, c2<T> b)
{
    T d = b.x * b.x + b.y * b.y;
    return mk<T>((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
template <class T> __device__ __forceinline__ c2<T> from_d(double2 a) { return mk<T>((T)a.x, (T)a.y); }

// ---------------------------------------------------------------------------------------------
// y = A_sign x:  y_a = (S + sign i tau H0)_{kappa_a} x_a - sign sum_{b>a} W_ab x_b + sign sum_{b<a} W_ba^T x_b
// one thread per (channel, radial slot), both DKB types; epilogues y <- bsub - y, partials <dv, y>,
// ||y||^2 (summed in double).
// ---------------------------------------------------------------------------------------------
template <class T, int BD>
__global__ void __launch_bounds__(128) k_apply(OpView A, const T* __restrict__ S, const T* __restrict__ H, int sign,
                                                const c2<T>* __restrict__ x, const T* __restrict__ W,
                                                c2<T>* __restrict__ y, const c2<T>* __restrict__ bsub,
                                                const c2<T>* __restrict__ dv, double2* part_dot, double* part_nrm,
                                                const KState* skip)
{
    if (skip && skip->done) return;   // uniform over the grid: the solve already finished
    const int bd = BD > 0 ? BD : A.bd;
    const int half = (bd - 1) / 2;
    const int n1 = A.n1;
    int ch = blockIdx.y;
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    c2<T> y0 = mk<T>(0, 0), y1 = mk<T>(0, 0);
    bool act = r < n1;
    if (act) {
        const c2<T>* xa = x + (int64_t)ch * 2 * n1;
        int ks = A.ch_kslot[ch];
        const T* Sk = S + ((int64_t)ks * n1 + r) * bd * 4;
        const T* Hk = H + ((int64_t)ks * n1 + r) * bd * 4;
        T st = (T)(sign * A.tau);
#pragma unroll
        for (int d = 0; d < bd; d++) {
            int rr = r + d - half;
            if (rr < 0 || rr >= n1) continue;
            c2<T> x0 = xa[2 * rr], x1 = xa[2 * rr + 1];
            T s00 = Sk[d * 4], s01 = Sk[d * 4 + 1], s10 = Sk[d * 4 + 2], s11 = Sk[d * 4 + 3];
            T h00 = st * Hk[d * 4], h01 = st * Hk[d * 4 + 1], h10 = st * Hk[d * 4 + 2], h11 = st * Hk[d * 4 + 3];
            y0.x += s00 * x0.x + s01 * x1.x - (h00 * x0.y + h01 * x1.y);
            y0.y += s00 * x0.y + s01 * x1.y + (h00 * x0.x + h01 * x1.x);
            y1.x += s10 * x0.x + s11 * x1.x - (h10 * x0.y + h11 * x1.y);
            y1.y += s10 * x0.y + s11 * x1.y + (h10 * x0.x + h11 * x1.x);
        }
        for (int e = A.adj_start[ch]; e < A.adj_start[ch + 1]; e++) {
            int64_t p = A.adj_pair[e];
            const c2<T>* xb = x + (int64_t)A.adj_nbr[e] * 2 * n1;
            const T* Wp = W + p * n1 * bd * 4;
            if (!A.adj_tr[e]) {
                T cs = (T)(-sign);
                const T* Wr = Wp + (int64_t)r * bd * 4;
#pragma unroll
                for (int d = 0; d < bd; d++) {
                    int rr = r + d - half;
                    if (rr < 0 || rr >= n1) continue;
                    c2<T> x0 = xb[2 * rr], x1 = xb[2 * rr + 1];
                    c2<T> wa = *reinterpret_cast<const c2<T>*>(Wr + d * 4);
                    c2<T> wb = *reinterpret_cast<const c2<T>*>(Wr + d * 4 + 2);
                    y0.x += cs * (wa.x * x0.x + wa.y * x1.x);
                    y0.y += cs * (wa.x * x0.y + wa.y * x1.y);
                    y1.x += cs * (wb.x * x0.x + wb.y * x1.x);
                    y1.y += cs * (wb.x * x0.y + wb.y * x1.y);
                }
            } else {
                T cs = (T)sign;
#pragma unroll
                for (int d = 0; d < bd; d++) {
                    int rr = r + d - half;
                    if (rr < 0 || rr >= n1) continue;
                    c2<T> x0 = xb[2 * rr], x1 = xb[2 * rr + 1];
                    const T* Wt = Wp + ((int64_t)rr * bd + (2 * half - d)) * 4;
                    c2<T> wa = *reinterpret_cast<const c2<T>*>(Wt);
                    c2<T> wb = *reinterpret_cast<const c2<T>*>(Wt + 2);
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
            c2<T> b0 = bsub[o], b1 = bsub[o + 1];
            y0 = mk<T>(b0.x - y0.x, b0.y - y0.y);
            y1 = mk<T>(b1.x - y1.x, b1.y - y1.y);
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
                c2<T> a = dv[o], b = dv[o + 1];
                dsum.x = (double)a.x * y0.x + (double)a.y * y0.y + (double)b.x * y1.x + (double)b.y * y1.y;
                dsum.y = (double)a.x * y0.y - (double)a.y * y0.x + (double)b.x * y1.y - (double)b.y * y1.x;
            }
            nsum = (double)y0.x * y0.x + (double)y0.y * y0.y + (double)y1.x * y1.x + (double)y1.y * y1.y;
        }
        block_reduce_store(dsum, nsum, part_dot, part_nrm, (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
    }
}

template <class T>
void launch_apply_t(dim3 grid, cudaStream_t st, const OpView& A, const T* S, const T* H, int sign, const void* x,
                    const T* W, void* y, const void* bsub, const void* dv, double2* pdot, double* pnrm,
                    const KState* skip)
{
    auto xx = (const c2<T>*)x;
    auto yy = (c2<T>*)y;
    auto bb = (const c2<T>*)bsub;
    auto dd = (const c2<T>*)dv;
    if (A.bd == 13)
        k_apply<T, 13><<<grid, 128, 0, st>>>(A, S, H, sign, xx, W, yy, bb, dd, pdot, pnrm, skip);
    else
        k_apply<T, 0><<<grid, 128, 0, st>>>(A, S, H, sign, xx, W, yy, bb, dd, pdot, pnrm, skip);
}

template void launch_apply_t<double>(dim3, cudaStream_t, const OpView&, const double*, const double*, int,
                                     const void*, const double*, void*, const void*, const void*, double2*,
                                     double*, const KState*);
template void launch_apply_t<float>(dim3, cudaStream_t, const OpView&, const float*, const float*, int, const void*,
                                    const float*, void*, const void*, const void*, double2*, double*, const KState*);

// ---------------------------------------------------------------------------------------------
// Preconditioner z = M^-1 v (Eq. matrixM), block diagonal over channels, one LU per kappa.
// One thread per channel: forward substitution with the recorded row interchanges, then back
// substitution.  Fused prologues (BiCGSTAB):
//   mode 0: v = r;   mode 1: p = r + beta (p - omega v) (stored in io);
//   mode 2: s = r - alpha v (stored in io, partial ||s||^2 in double).
// ---------------------------------------------------------------------------------------------
template <class T>
__global__ void k_precond(OpView A, const c2<T>* __restrict__ U, const c2<T>* __restrict__ L, int mode,
                          const KState* st, const c2<T>* __restrict__ r, const c2<T>* __restrict__ v,
                          c2<T>* __restrict__ io, c2<T>* __restrict__ z, double* part_nrm)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    double nsum = 0;
    if (idx < A.nch && !(st && st->done)) {
        int ch = A.prec_order[idx];
        int n = 2 * A.n1, kb = A.kb, wu = 2 * kb;
        int ks = A.ch_kslot[ch];
        const c2<T>* Uk = U + (int64_t)ks * n * (wu + 1);
        const c2<T>* Lk = L + (int64_t)ks * n * kb;
        const int* P = A.luP + (int64_t)ks * n;
        int64_t o = (int64_t)ch * n;
        c2<T>* zc = z + o;
        if (mode == 0) {
            for (int i = 0; i < n; i++) zc[i] = r[o + i];
        } else if (mode == 1) {
            c2<T> beta = from_d<T>(st->beta), omega = from_d<T>(st->omega);
            for (int i = 0; i < n; i++) {
                c2<T> pv = io[o + i], vv = v[o + i], rv = r[o + i];
                c2<T> t = cm<T>(omega, vv);
                c2<T> q = cm<T>(beta, mk<T>(pv.x - t.x, pv.y - t.y));
                c2<T> pn = mk<T>(rv.x + q.x, rv.y + q.y);
                io[o + i] = pn;
                zc[i] = pn;
            }
        } else {
            c2<T> alpha = from_d<T>(st->alpha);
            for (int i = 0; i < n; i++) {
                c2<T> t = cm<T>(alpha, v[o + i]);
                c2<T> rv = r[o + i];
                c2<T> sv = mk<T>(rv.x - t.x, rv.y - t.y);
                io[o + i] = sv;
                zc[i] = sv;
                nsum += (double)sv.x * sv.x + (double)sv.y * sv.y;
            }
        }
        for (int j = 0; j < n; j++) {
            int pj = P[j];
            if (pj != j) { c2<T> t = zc[j]; zc[j] = zc[pj]; zc[pj] = t; }
            c2<T> zj = zc[j];
            int lim = min(kb, n - 1 - j);
            for (int i = 1; i <= lim; i++) {
                c2<T> m = cm<T>(Lk[(int64_t)j * kb + i - 1], zj);
                zc[j + i].x -= m.x;
                zc[j + i].y -= m.y;
            }
        }
        for (int i = n - 1; i >= 0; i--) {
            c2<T> s = zc[i];
            int lim = min(wu, n - 1 - i);
            const c2<T>* Ui = Uk + (int64_t)i * (wu + 1);
            for (int k = 1; k <= lim; k++) {
                c2<T> m = cm<T>(Ui[k], zc[i + k]);
                s.x -= m.x;
                s.y -= m.y;
            }
            zc[i] = cdv<T>(s, Ui[0]);
        }
    }
    if (part_nrm) block_reduce_store(make_double2(0, 0), nsum, nullptr, part_nrm, blockIdx.x);
}

template <class T>
void launch_precond_t(int blocks, cudaStream_t st, const OpView& A, const void* U, const void* L, int mode,
                      const KState* ks, const void* r, const void* v, void* io, void* z, double* pn)
{
    k_precond<T><<<blocks, 32, 0, st>>>(A, (const c2<T>*)U, (const c2<T>*)L, mode, ks, (const c2<T>*)r,
                                        (const c2<T>*)v, (c2<T>*)io, (c2<T>*)z, pn);
}
template void launch_precond_t<double>(int, cudaStream_t, const OpView&, const void*, const void*, int,
                                       const KState*, const void*, const void*, void*, void*, double*);
template void launch_precond_t<float>(int, cudaStream_t, const OpView&, const void*, const void*, int,
                                      const KState*, const void*, const void*, void*, void*, double*);

// ---------------------------------------------------------------------------------------------
// x += alpha ph + omega sh;  r = s - omega t;  partials <rh, r>, ||r||^2.  After the s-check ended
// the solve (done == 2): x += alpha ph only.
// ---------------------------------------------------------------------------------------------
template <class T>
__global__ void k_update_xr(int64_t n, const KState* st, c2<T>* x, c2<T>* r, const c2<T>* ph, const c2<T>* sh,
                            const c2<T>* s, const c2<T>* t, const c2<T>* rh, double2* part_dot, double* part_nrm)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double2 dsum = make_double2(0, 0);
    double nsum = 0;
    if (i < n && st->status == 0) {
        c2<T> a = cm<T>(from_d<T>(st->alpha), ph[i]);
        if (st->done == 2) {
            x[i].x += a.x;
            x[i].y += a.y;
        } else if (!st->done) {
            c2<T> w = cm<T>(from_d<T>(st->omega), sh[i]);
            x[i].x += a.x + w.x;
            x[i].y += a.y + w.y;
            c2<T> ot = cm<T>(from_d<T>(st->omega), t[i]);
            c2<T> rn = mk<T>(s[i].x - ot.x, s[i].y - ot.y);
            r[i] = rn;
            c2<T> h = rh[i];
            dsum.x = (double)h.x * rn.x + (double)h.y * rn.y;
            dsum.y = (double)h.x * rn.y - (double)h.y * rn.x;
            nsum = (double)rn.x * rn.x + (double)rn.y * rn.y;
        }
    }
    block_reduce_store(dsum, nsum, part_dot, part_nrm, blockIdx.x);
}

template <class T>
void launch_update_xr_t(int blocks, cudaStream_t st, int64_t n, const KState* ks, void* x, void* r, const void* ph,
                        const void* sh, const void* s, const void* t, const void* rh, double2* pd, double* pn)
{
    k_update_xr<T><<<blocks, 256, 0, st>>>(n, ks, (c2<T>*)x, (c2<T>*)r, (const c2<T>*)ph, (const c2<T>*)sh,
                                           (const c2<T>*)s, (const c2<T>*)t, (const c2<T>*)rh, pd, pn);
}
template void launch_update_xr_t<double>(int, cudaStream_t, int64_t, const KState*, void*, void*, const void*,
                                         const void*, const void*, const void*, const void*, double2*, double*);
template void launch_update_xr_t<float>(int, cudaStream_t, int64_t, const KState*, void*, void*, const void*,
                                        const void*, const void*, const void*, const void*, double2*, double*);

// ---------------------------------------------------------------------------------------------
// Precision conversions of the refinement loop: d32 = r64 / ||r|| (scaled inner right-hand side)
// and x64 += ||r|| d32.  scale_src holds ||r||^2 (the outer KState's rnorm2).
// ---------------------------------------------------------------------------------------------
__global__ void k_to_float_scaled(int64_t n, const double2* a, const KState* st, float2* b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = st->rnorm2 > 0 ? 1.0 / sqrt(st->rnorm2) : 0.0;
    b[i] = make_float2((float)(a[i].x * s), (float)(a[i].y * s));
}

__global__ void k_add_float_scaled(int64_t n, const float2* d, const KState* st, double2* x)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = sqrt(st->rnorm2);
    x[i].x += s * (double)d[i].x;
    x[i].y += s * (double)d[i].y;
}

__global__ void k_copy32(int64_t n, const float2* a, float2* b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

__global__ void k_zero32(int64_t n, float2* a)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = make_float2(0, 0);
}

}  // namespace dg
