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
    // tile-major order (all channels of one radial tile, then the next tile): both uses of a
    // coupling block (W x_b by its lower channel, W^T x_a by its upper one) fall in the same tile
    // slab of the coupling values, which fits in L2, so the block is read from HBM once
    int ch = blockIdx.x;
    int r = blockIdx.y * blockDim.x + threadIdx.x;
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
        // coupling: direct (W x) and transposed (W^T x) sums kept apart so every stored value costs
        // exactly two FMAs per use; the signs are applied once at the end
        c2<T> d0 = mk<T>(0, 0), d1 = mk<T>(0, 0), t0 = mk<T>(0, 0), t1 = mk<T>(0, 0);
        for (int e = A.adj_start[ch]; e < A.adj_start[ch + 1]; e++) {
            int64_t p = A.adj_pair[e];
            const c2<T>* xb = x + (int64_t)A.adj_nbr[e] * 2 * n1;
            const T* Wp = W + p * n1 * bd * 4;
            if (!A.adj_tr[e]) {
                const T* Wr = Wp + (int64_t)r * bd * 4;
#pragma unroll
                for (int d = 0; d < bd; d++) {
                    int rr = r + d - half;
                    if (rr < 0 || rr >= n1) continue;
                    c2<T> x0 = xb[2 * rr], x1 = xb[2 * rr + 1];
                    c2<T> wa = *reinterpret_cast<const c2<T>*>(Wr + d * 4);
                    c2<T> wb = *reinterpret_cast<const c2<T>*>(Wr + d * 4 + 2);
                    d0.x = fma(wa.x, x0.x, d0.x); d0.x = fma(wa.y, x1.x, d0.x);
                    d0.y = fma(wa.x, x0.y, d0.y); d0.y = fma(wa.y, x1.y, d0.y);
                    d1.x = fma(wb.x, x0.x, d1.x); d1.x = fma(wb.y, x1.x, d1.x);
                    d1.y = fma(wb.x, x0.y, d1.y); d1.y = fma(wb.y, x1.y, d1.y);
                }
            } else {
#pragma unroll
                for (int d = 0; d < bd; d++) {
                    int rr = r + d - half;
                    if (rr < 0 || rr >= n1) continue;
                    c2<T> x0 = xb[2 * rr], x1 = xb[2 * rr + 1];
                    const T* Wt = Wp + ((int64_t)rr * bd + (2 * half - d)) * 4;
                    c2<T> wa = *reinterpret_cast<const c2<T>*>(Wt);
                    c2<T> wb = *reinterpret_cast<const c2<T>*>(Wt + 2);
                    // (W^T)[t][u] = W[u][t]
                    t0.x = fma(wa.x, x0.x, t0.x); t0.x = fma(wb.x, x1.x, t0.x);
                    t0.y = fma(wa.x, x0.y, t0.y); t0.y = fma(wb.x, x1.y, t0.y);
                    t1.x = fma(wa.y, x0.x, t1.x); t1.x = fma(wb.y, x1.x, t1.x);
                    t1.y = fma(wa.y, x0.y, t1.y); t1.y = fma(wb.y, x1.y, t1.y);
                }
            }
        }
        // y += sign (sum W^T x - sum W x)
        T sg = (T)sign;
        y0.x = fma(sg, t0.x - d0.x, y0.x); y0.y = fma(sg, t0.y - d0.y, y0.y);
        y1.x = fma(sg, t1.x - d1.x, y1.x); y1.y = fma(sg, t1.y - d1.y, y1.y);
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
// Preconditioner z = M^-1 v (Eq. matrixM), block diagonal over channels, one banded LU per kappa.
// One warp per channel (channels sorted by kappa, so neighbouring warps share factors):
//  - prologue, lanes over the vector:  mode 0: v = r;  mode 1: p = r + beta (p - omega v) (kept in
//    io);  mode 2: s = r - alpha v (kept in io; partial ||s||^2 summed in double);
//  - forward substitution column by column: lanes 0..kb hold z[j..j+kb]; the recorded row
//    interchange of column j swaps lane 0 with lane piv[j]-j, lanes 1..kb subtract L[j] z[j],
//    then the window slides by one;
//  - back substitution column by column: lane k accumulates U[i-k][k] x[i] for row i-k, so row i
//    is complete when it reaches lane 1 and no per-row reduction is needed.  Ucol[i][k] = U[i-k][k].
// ---------------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ c2<T> shfl2(c2<T> v, int src)
{
    return mk<T>(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
template <class T>
__device__ __forceinline__ c2<T> shfl2_down(c2<T> v, int d)
{
    return mk<T>(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

template <class T>
__global__ void __launch_bounds__(128) k_precond(OpView A, const c2<T>* __restrict__ Ucol,
                                                 const c2<T>* __restrict__ L, const c2<T>* __restrict__ Dinv,
                                                 int mode, const KState* st,
                                                 const c2<T>* __restrict__ r, const c2<T>* __restrict__ v,
                                                 c2<T>* __restrict__ io, c2<T>* __restrict__ z, double* part_nrm)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    double nsum = 0;
    if (warp < A.nch && !(st && st->done)) {
        int ch = A.prec_order[warp];
        const int n = 2 * A.n1, kb = A.kb, wu = 2 * kb;
        int ks = A.ch_kslot[ch];
        const c2<T>* Uk = Ucol + (int64_t)ks * n * (wu + 1);
        const c2<T>* Lk = L + (int64_t)ks * n * kb;
        const c2<T>* Dk = Dinv + (int64_t)ks * n;
        const int* P = A.luP + (int64_t)ks * n;
        int64_t o = (int64_t)ch * n;
        c2<T>* zc = z + o;
        if (mode == 0) {
            for (int i = lane; i < n; i += 32) zc[i] = r[o + i];
        } else if (mode == 1) {
            c2<T> beta = from_d<T>(st->beta), omega = from_d<T>(st->omega);
            for (int i = lane; i < n; i += 32) {
                c2<T> pv = io[o + i], vv = v[o + i], rv = r[o + i];
                c2<T> t = cm<T>(omega, vv);
                c2<T> q = cm<T>(beta, mk<T>(pv.x - t.x, pv.y - t.y));
                c2<T> pn = mk<T>(rv.x + q.x, rv.y + q.y);
                io[o + i] = pn;
                zc[i] = pn;
            }
        } else {
            c2<T> alpha = from_d<T>(st->alpha);
            for (int i = lane; i < n; i += 32) {
                c2<T> t = cm<T>(alpha, v[o + i]);
                c2<T> rv = r[o + i];
                c2<T> sv = mk<T>(rv.x - t.x, rv.y - t.y);
                io[o + i] = sv;
                zc[i] = sv;
                nsum += (double)sv.x * sv.x + (double)sv.y * sv.y;
            }
        }
        __syncwarp();
        // forward: window lane l = z[j + l], l = 0..kb; row j + 1 of L and its pivot loaded ahead
        c2<T> w = (lane <= kb && lane < n) ? zc[lane] : mk<T>(0, 0);
        c2<T> lnext = (lane >= 1 && lane <= kb) ? Lk[lane - 1] : mk<T>(0, 0);
        int pnext = P[0];
        for (int j = 0; j < n; j++) {
            c2<T> lcur = lnext;
            int pj = pnext - j;
            if (j + 1 < n) {
                lnext = (lane >= 1 && lane <= kb) ? Lk[(int64_t)(j + 1) * kb + lane - 1] : mk<T>(0, 0);
                pnext = P[j + 1];
            }
            c2<T> w0 = shfl2<T>(w, 0), wp = shfl2<T>(w, pj);
            if (lane == 0) w = wp;
            else if (lane == pj) w = w0;
            c2<T> zj = shfl2<T>(w, 0);
            if (lane >= 1 && lane <= kb && j + lane < n) {
                w.x -= lcur.x * zj.x - lcur.y * zj.y;
                w.y -= lcur.x * zj.y + lcur.y * zj.x;
            }
            if (lane == 0) zc[j] = zj;
            w = shfl2_down<T>(w, 1);
            if (lane == kb) w = (j + kb + 1 < n) ? zc[j + kb + 1] : mk<T>(0, 0);
        }
        __syncwarp();
        // backward: lane k (1..wu) holds the partial sum of row i - k; the row of U for the next
        // step is loaded one step ahead
        c2<T> acc = mk<T>(0, 0);
        c2<T> unext = (lane >= 1 && lane <= wu && n - 1 - lane >= 0) ? Uk[(int64_t)(n - 1) * (wu + 1) + lane]
                                                                      : mk<T>(0, 0);
        for (int i = n - 1; i >= 0; i--) {
            c2<T> ucur = unext;
            if (i > 0) unext = (lane >= 1 && lane <= wu && i - 1 - lane >= 0) ? Uk[(int64_t)(i - 1) * (wu + 1) + lane]
                                                                              : mk<T>(0, 0);
            // row i is complete in lane 1; lane 0 finishes it with the reciprocal diagonal
            c2<T> a0 = shfl2<T>(acc, 1);
            c2<T> xi = mk<T>(0, 0);
            if (lane == 0) {
                c2<T> zi = zc[i];
                xi = cm<T>(mk<T>(zi.x - a0.x, zi.y - a0.y), Dk[i]);
                zc[i] = xi;
            }
            xi = shfl2<T>(xi, 0);
            // slide: lane k takes the sum of row (i-1) - k from lane k + 1, then adds U[i-k][k] x[i]
            acc = shfl2_down<T>(acc, 1);
            if (lane == wu) acc = mk<T>(0, 0);
            if (lane >= 1 && lane <= wu) {
                acc.x += ucur.x * xi.x - ucur.y * xi.y;
                acc.y += ucur.x * xi.y + ucur.y * xi.x;
            }
        }
    }
    if (part_nrm) {
        // per-block partial of ||s||^2 (one value per block in a fixed order)
        block_reduce_store(make_double2(0, 0), nsum, nullptr, part_nrm, blockIdx.x);
    }
}

// Lane-per-channel variant for band width 13 (order-7 B-splines): one warp per group of <= 32
// channels of the same kappa (warp_ks, warp_first, warp_count), so factor loads are broadcasts
// and the recorded interchanges are warp-uniform.  Each lane runs the whole substitution of its
// channel with the windows in registers: forward z[j..j+13], backward x[i+1..i+26]; the diagonal
// of U is applied as a precomputed reciprocal.  Urow[i][k] = U[i][i+k].
template <class T, int KB>
__global__ void __launch_bounds__(32) k_precond_lanes(OpView A, const c2<T>* __restrict__ Urow,
                                                      const c2<T>* __restrict__ L, const c2<T>* __restrict__ Dinv,
                                                      const int* __restrict__ warp_ks, const int* __restrict__ warp_first,
                                                      const int* __restrict__ warp_count, int mode, const KState* st,
                                                      const c2<T>* __restrict__ r, const c2<T>* __restrict__ v,
                                                      c2<T>* __restrict__ io, c2<T>* __restrict__ z, double* part_nrm)
{
    constexpr int WU = 2 * KB;
    int w = blockIdx.x, lane = threadIdx.x;
    double nsum = 0;
    if (!(st && st->done)) {
        const int n = 2 * A.n1;
        int ks = warp_ks[w], first = warp_first[w], cnt = warp_count[w];
        // prologue, coalesced: lanes over the entries of each channel of the group
        for (int c = 0; c < cnt; c++) {
            int64_t o = (int64_t)A.prec_order[first + c] * n;
            if (mode == 0) {
                for (int i = lane; i < n; i += 32) z[o + i] = r[o + i];
            } else if (mode == 1) {
                c2<T> beta = from_d<T>(st->beta), omega = from_d<T>(st->omega);
                for (int i = lane; i < n; i += 32) {
                    c2<T> pv = io[o + i], vv = v[o + i], rv = r[o + i];
                    c2<T> t = cm<T>(omega, vv);
                    c2<T> q = cm<T>(beta, mk<T>(pv.x - t.x, pv.y - t.y));
                    c2<T> pn = mk<T>(rv.x + q.x, rv.y + q.y);
                    io[o + i] = pn;
                    z[o + i] = pn;
                }
            } else {
                c2<T> alpha = from_d<T>(st->alpha);
                for (int i = lane; i < n; i += 32) {
                    c2<T> t = cm<T>(alpha, v[o + i]);
                    c2<T> rv = r[o + i];
                    c2<T> sv = mk<T>(rv.x - t.x, rv.y - t.y);
                    io[o + i] = sv;
                    z[o + i] = sv;
                    nsum += (double)sv.x * sv.x + (double)sv.y * sv.y;
                }
            }
        }
        __syncwarp();
        // factor rows are staged through shared memory CH rows at a time (one coalesced load per
        // chunk, then broadcast reads); the rows are the same for every lane (same kappa)
        constexpr int CH = 32;
        __shared__ c2<T> sF[CH * (WU + 1)];
        __shared__ c2<T> sD[CH];
        __shared__ int sP[CH];
        const bool mine = lane < cnt;
        int64_t o = mine ? (int64_t)A.prec_order[first + lane] * n : 0;
        c2<T>* zc = z + o;
        const c2<T>* Lk = L + (int64_t)ks * n * KB;
        const c2<T>* Uk = Urow + (int64_t)ks * n * (WU + 1);
        const c2<T>* Dk = Dinv + (int64_t)ks * n;
        const int* P = A.luP + (int64_t)ks * n;
        c2<T> win[KB + 1];
#pragma unroll
        for (int i = 0; i <= KB; i++) win[i] = (mine && i < n) ? zc[i] : mk<T>(0, 0);
        for (int j0 = 0; j0 < n; j0 += CH) {
            int rows = min(CH, n - j0);
            __syncwarp();
            for (int e = lane; e < rows * KB; e += 32) sF[e] = Lk[(int64_t)j0 * KB + e];
            if (lane < rows) sP[lane] = P[j0 + lane];
            __syncwarp();
            if (mine)
                for (int jj = 0; jj < rows; jj++) {
                    int j = j0 + jj;
                    int pj = sP[jj] - j;
#pragma unroll
                    for (int i = 1; i <= KB; i++)
                        if (pj == i) { c2<T> t = win[0]; win[0] = win[i]; win[i] = t; }
                    c2<T> zj = win[0];
                    zc[j] = zj;
#pragma unroll
                    for (int i = 1; i <= KB; i++) {
                        c2<T> l = sF[jj * KB + i - 1];   // zero beyond the last row
                        win[i].x -= l.x * zj.x - l.y * zj.y;
                        win[i].y -= l.x * zj.y + l.y * zj.x;
                    }
#pragma unroll
                    for (int i = 0; i < KB; i++) win[i] = win[i + 1];
                    win[KB] = (j + KB + 1 < n) ? zc[j + KB + 1] : mk<T>(0, 0);
                }
        }
        c2<T> xw[WU];
#pragma unroll
        for (int k = 0; k < WU; k++) xw[k] = mk<T>(0, 0);
        c2<T> znext = mine ? zc[n - 1] : mk<T>(0, 0);
        for (int i1 = n - 1; i1 >= 0; i1 -= CH) {
            int rows = min(CH, i1 + 1);   // rows i1 - rows + 1 .. i1
            int i0 = i1 - rows + 1;
            __syncwarp();
            for (int e = lane; e < rows * (WU + 1); e += 32) sF[e] = Uk[(int64_t)i0 * (WU + 1) + e];
            if (lane < rows) sD[lane] = Dk[i0 + lane];
            __syncwarp();
            if (mine)
                for (int ii = rows - 1; ii >= 0; ii--) {
                    int i = i0 + ii;
                    c2<T> s = znext;
                    if (i > 0) znext = zc[i - 1];
                    const c2<T>* Ui = sF + ii * (WU + 1);
#pragma unroll
                    for (int k = 1; k <= WU; k++) {
                        c2<T> u = Ui[k];       // zero beyond the last column
                        s.x -= u.x * xw[k - 1].x - u.y * xw[k - 1].y;
                        s.y -= u.x * xw[k - 1].y + u.y * xw[k - 1].x;
                    }
                    c2<T> xi = cm<T>(s, sD[ii]);
                    zc[i] = xi;
#pragma unroll
                    for (int k = WU - 1; k > 0; k--) xw[k] = xw[k - 1];
                    xw[0] = xi;
                }
        }
    }
    if (part_nrm) block_reduce_store(make_double2(0, 0), nsum, nullptr, part_nrm, blockIdx.x);
}

template <class T>
void launch_precond_lanes_t(int nwarps, cudaStream_t st, const OpView& A, const void* Urow, const void* L,
                            const void* Dinv, const int* wks, const int* wfirst, const int* wcnt, int mode,
                            const KState* ks, const void* r, const void* v, void* io, void* z, double* pn)
{
    k_precond_lanes<T, 13><<<nwarps, 32, 0, st>>>(A, (const c2<T>*)Urow, (const c2<T>*)L, (const c2<T>*)Dinv, wks,
                                                  wfirst, wcnt, mode, ks, (const c2<T>*)r, (const c2<T>*)v,
                                                  (c2<T>*)io, (c2<T>*)z, pn);
}
template void launch_precond_lanes_t<double>(int, cudaStream_t, const OpView&, const void*, const void*,
                                             const void*, const int*, const int*, const int*, int, const KState*,
                                             const void*, const void*, void*, void*, double*);
template void launch_precond_lanes_t<float>(int, cudaStream_t, const OpView&, const void*, const void*, const void*,
                                            const int*, const int*, const int*, int, const KState*, const void*,
                                            const void*, void*, void*, double*);

template <class T>
void launch_precond_t(int blocks, cudaStream_t st, const OpView& A, const void* U, const void* L, const void* Dinv,
                      int mode, const KState* ks, const void* r, const void* v, void* io, void* z, double* pn)
{
    k_precond<T><<<blocks, 128, 0, st>>>(A, (const c2<T>*)U, (const c2<T>*)L, (const c2<T>*)Dinv, mode, ks,
                                         (const c2<T>*)r, (const c2<T>*)v, (c2<T>*)io, (c2<T>*)z, pn);
}
template void launch_precond_t<double>(int, cudaStream_t, const OpView&, const void*, const void*, const void*, int,
                                       const KState*, const void*, const void*, void*, void*, double*);
template void launch_precond_t<float>(int, cudaStream_t, const OpView&, const void*, const void*, const void*, int,
                                      const KState*, const void*, const void*, void*, void*, double*);

// ---------------------------------------------------------------------------------------------
// Warp-per-channel preconditioner with the channel's vector in shared memory and the factor rows
// staged through shared memory in chunks of CH rows by asynchronous copies (cp.async), one chunk
// ahead.  The substitution is the same as k_precond (same operations in the same order, so the
// results are identical); what changes is where the operands come from: every row of the sweeps
// reads shared memory instead of waiting on an L2 load.  Band width KB = 13 (order-7 splines).
// ---------------------------------------------------------------------------------------------
namespace {
constexpr int PCH = 16;   // factor rows per staged chunk

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// copy `bytes` (a multiple of 16, both addresses 16-byte aligned) with the warp's lanes
__device__ __forceinline__ void warp_copy16(void* dst, const void* src, int bytes, int lane)
{
    for (int e = lane; e < bytes / 16; e += 32)
        cp_async16(static_cast<char*>(dst) + 16 * e, static_cast<const char*>(src) + 16 * e);
}
}  // namespace

template <class T>
constexpr int prec_sm_warps() { return sizeof(T) == 4 ? 4 : 2; }

// per-warp shared memory: the vector (n entries) and the factor chunk buffers
template <class T, int KB>
__host__ __device__ constexpr size_t prec_sm_fbytes()
{
    // forward: L[2][PCH][KB] + P[2][PCH] (ints); backward: Ucol[2][PCH][2 KB + 1] + Dinv[2][PCH]
    return sizeof(c2<T>) * (2 * PCH * (2 * KB + 1) + 2 * PCH) > sizeof(c2<T>) * 2 * PCH * KB + 2 * PCH * 4
               ? sizeof(c2<T>) * (2 * PCH * (2 * KB + 1) + 2 * PCH)
               : sizeof(c2<T>) * 2 * PCH * KB + 2 * PCH * 4;
}
template <class T, int KB>
size_t prec_sm_warp_bytes(int n)
{
    return ((sizeof(c2<T>) * (size_t)n + 15) / 16) * 16 + prec_sm_fbytes<T, KB>();
}

template <class T, int KB>
__global__ void k_precond_sm(OpView A, const c2<T>* __restrict__ Ucol, const c2<T>* __restrict__ L,
                             const c2<T>* __restrict__ Dinv, int mode, const KState* st,
                             const c2<T>* __restrict__ r, const c2<T>* __restrict__ v, c2<T>* __restrict__ io,
                             c2<T>* __restrict__ z, double* part_nrm, int warp_bytes)
{
    constexpr int WU = 2 * KB;
    extern __shared__ __align__(16) unsigned char prec_smem[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
    const int n = 2 * A.n1;
    unsigned char* base = prec_smem + (size_t)wib * warp_bytes;
    c2<T>* zs = reinterpret_cast<c2<T>*>(base);
    unsigned char* fb = base + ((sizeof(c2<T>) * (size_t)n + 15) / 16) * 16;
    c2<T>* Lb = reinterpret_cast<c2<T>*>(fb);                          // [2][PCH * KB]
    int* Pb = reinterpret_cast<int*>(fb + sizeof(c2<T>) * 2 * PCH * KB);  // [2][PCH]
    c2<T>* Ub = reinterpret_cast<c2<T>*>(fb);                          // [2][PCH * (WU + 1)]
    c2<T>* Db = Ub + 2 * PCH * (WU + 1);                               // [2][PCH]
    double nsum = 0;
    if (warp < A.nch && !(st && st->done)) {
        const int ch = A.prec_order[warp];
        const int ks = A.ch_kslot[ch];
        const c2<T>* Uk = Ucol + (int64_t)ks * n * (WU + 1);
        const c2<T>* Lk = L + (int64_t)ks * n * KB;
        const c2<T>* Dk = Dinv + (int64_t)ks * n;
        const int* P = A.luP + (int64_t)ks * n;
        const int64_t o = (int64_t)ch * n;
        // forward factor chunk c into buffer b: rows [c PCH, c PCH + rows)
        auto issue_fwd = [&](int c, int b) {
            int j0 = c * PCH, rows = min(PCH, n - j0);
            warp_copy16(Lb + b * PCH * KB, Lk + (int64_t)j0 * KB, rows * KB * (int)sizeof(c2<T>), lane);
            for (int e = lane; e < rows; e += 32) cp_async4(Pb + b * PCH + e, P + j0 + e);
            cp_async_commit();
        };
        issue_fwd(0, 0);
        // prologue into the shared copy of the vector
        if (mode == 0) {
            for (int i = lane; i < n; i += 32) zs[i] = r[o + i];
        } else if (mode == 1) {
            c2<T> beta = from_d<T>(st->beta), omega = from_d<T>(st->omega);
            for (int i = lane; i < n; i += 32) {
                c2<T> pv = io[o + i], vv = v[o + i], rv = r[o + i];
                c2<T> t = cm<T>(omega, vv);
                c2<T> q = cm<T>(beta, mk<T>(pv.x - t.x, pv.y - t.y));
                c2<T> pn = mk<T>(rv.x + q.x, rv.y + q.y);
                io[o + i] = pn;
                zs[i] = pn;
            }
        } else {
            c2<T> alpha = from_d<T>(st->alpha);
            for (int i = lane; i < n; i += 32) {
                c2<T> t = cm<T>(alpha, v[o + i]);
                c2<T> rv = r[o + i];
                c2<T> sv = mk<T>(rv.x - t.x, rv.y - t.y);
                io[o + i] = sv;
                zs[i] = sv;
                nsum += (double)sv.x * sv.x + (double)sv.y * sv.y;
            }
        }
        __syncwarp();
        // forward substitution: window lane l = z[j + l], l = 0..KB
        c2<T> w = (lane <= KB && lane < n) ? zs[lane] : mk<T>(0, 0);
        const int nc = (n + PCH - 1) / PCH;
        for (int c = 0; c < nc; c++) {
            if (c + 1 < nc) {
                issue_fwd(c + 1, (c + 1) & 1);
                cp_async_wait1();
            } else {
                cp_async_wait0();
            }
            __syncwarp();
            const c2<T>* Lc = Lb + (c & 1) * PCH * KB;
            const int* Pc = Pb + (c & 1) * PCH;
            const int j0 = c * PCH, rows = min(PCH, n - j0);
            for (int jj = 0; jj < rows; jj++) {
                const int j = j0 + jj;
                c2<T> lcur = (lane >= 1 && lane <= KB) ? Lc[jj * KB + lane - 1] : mk<T>(0, 0);
                int pj = Pc[jj] - j;
                c2<T> w0 = shfl2<T>(w, 0), wp = shfl2<T>(w, pj);
                if (lane == 0) w = wp;
                else if (lane == pj) w = w0;
                c2<T> zj = shfl2<T>(w, 0);
                if (lane >= 1 && lane <= KB && j + lane < n) {
                    w.x -= lcur.x * zj.x - lcur.y * zj.y;
                    w.y -= lcur.x * zj.y + lcur.y * zj.x;
                }
                if (lane == 0) zs[j] = zj;
                w = shfl2_down<T>(w, 1);
                if (lane == KB) w = (j + KB + 1 < n) ? zs[j + KB + 1] : mk<T>(0, 0);
            }
            __syncwarp();   // buffer (c & 1) is refilled by the next iteration's copy
        }
        // back substitution: lane k (1..WU) holds the partial sum of row i - k
        auto issue_bwd = [&](int c, int b) {
            int i0 = c * PCH, rows = min(PCH, n - i0);
            warp_copy16(Ub + b * PCH * (WU + 1), Uk + (int64_t)i0 * (WU + 1), rows * (WU + 1) * (int)sizeof(c2<T>), lane);
            warp_copy16(Db + b * PCH, Dk + i0, rows * (int)sizeof(c2<T>), lane);
            cp_async_commit();
        };
        issue_bwd(nc - 1, 0);
        c2<T> acc = mk<T>(0, 0);
        for (int q = 0; q < nc; q++) {
            const int c = nc - 1 - q;
            if (c > 0) {
                issue_bwd(c - 1, (q + 1) & 1);
                cp_async_wait1();
            } else {
                cp_async_wait0();
            }
            __syncwarp();
            const c2<T>* Uc = Ub + (q & 1) * PCH * (WU + 1);
            const c2<T>* Dc = Db + (q & 1) * PCH;
            const int i0 = c * PCH, rows = min(PCH, n - i0);
            for (int ii = rows - 1; ii >= 0; ii--) {
                const int i = i0 + ii;
                c2<T> ucur = (lane >= 1 && lane <= WU && i - lane >= 0) ? Uc[ii * (WU + 1) + lane] : mk<T>(0, 0);
                c2<T> a0 = shfl2<T>(acc, 1);
                c2<T> xi = mk<T>(0, 0);
                if (lane == 0) {
                    c2<T> zi = zs[i];
                    xi = cm<T>(mk<T>(zi.x - a0.x, zi.y - a0.y), Dc[ii]);
                    zs[i] = xi;
                }
                xi = shfl2<T>(xi, 0);
                acc = shfl2_down<T>(acc, 1);
                if (lane == WU) acc = mk<T>(0, 0);
                if (lane >= 1 && lane <= WU) {
                    acc.x += ucur.x * xi.x - ucur.y * xi.y;
                    acc.y += ucur.x * xi.y + ucur.y * xi.x;
                }
            }
            __syncwarp();
        }
        // result out, coalesced
        c2<T>* zc = z + o;
        for (int i = lane; i < n; i += 32) zc[i] = zs[i];
    }
    if (part_nrm) block_reduce_store(make_double2(0, 0), nsum, nullptr, part_nrm, blockIdx.x);
}

// ---------------------------------------------------------------------------------------------
// Rotated-lane form of the same substitutions: row r of the window lives in lane r mod 32 for
// its whole life, so the window never shifts.  A forward step j takes the pivot row's value with
// one shuffle (plus the row-j value for the interchange, in parallel), and the lanes of rows
// j+1..j+kb subtract L[j] z[j]; a backward step i forms x[i] in lane i mod 32 from its completed
// sum and broadcasts it with one shuffle to the lanes of rows i-1..i-2kb.  That is one shuffle
// round per row on the dependency chain (two in the shifting window).  The vector never lives
// whole in shared memory: 16-row chunks of the input (forward) and of the forward result
// (backward) arrive by cp.async together with the factor chunks, so a warp needs a few KB and
// every channel's warp is resident at once.  The forward result goes to z and comes back for the
// backward sweep.  Same arithmetic, in the same order, as the shifting-window kernels.
// ---------------------------------------------------------------------------------------------
template <class T>
constexpr int prec_rot_warps() { return sizeof(T) == 4 ? 4 : 2; }

constexpr int ROT_VRING = 4;   // vector chunks in flight per warp (forward input, backward z)

template <class T, int KB>
__host__ __device__ constexpr size_t prec_rot_warp_bytes()
{
    return prec_sm_fbytes<T, KB>() + sizeof(c2<T>) * ROT_VRING * PCH;
}

template <class T, int KB>
__global__ void k_precond_rot(OpView A, const c2<T>* __restrict__ Ucol, const c2<T>* __restrict__ L,
                              const c2<T>* __restrict__ Dinv, int mode, const KState* st,
                              const c2<T>* __restrict__ r, const c2<T>* __restrict__ v, c2<T>* __restrict__ io,
                              c2<T>* __restrict__ z, double* part_nrm)
{
    constexpr int WU = 2 * KB;
    static_assert(WU + 1 <= 32 && KB < PCH, "the windows must fit in a warp and reach one chunk ahead");
    extern __shared__ __align__(16) unsigned char prec_smem[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + wib;
    const int n = 2 * A.n1;
    unsigned char* fb = prec_smem + (size_t)wib * prec_rot_warp_bytes<T, KB>();
    c2<T>* Lb = reinterpret_cast<c2<T>*>(fb);                          // [2][PCH * KB]
    int* Pb = reinterpret_cast<int*>(fb + sizeof(c2<T>) * 2 * PCH * KB);  // [2][PCH]
    c2<T>* Ub = reinterpret_cast<c2<T>*>(fb);                          // [2][PCH * (WU + 1)]
    c2<T>* Db = Ub + 2 * PCH * (WU + 1);                               // [2][PCH]
    c2<T>* Vb = reinterpret_cast<c2<T>*>(fb + prec_sm_fbytes<T, KB>());  // [ROT_VRING][PCH]
    double nsum = 0;
    if (warp < A.nch && !(st && st->done)) {
        const int ch = A.prec_order[warp];
        const int ks = A.ch_kslot[ch];
        const c2<T>* Uk = Ucol + (int64_t)ks * n * (WU + 1);
        const c2<T>* Lk = L + (int64_t)ks * n * KB;
        const c2<T>* Dk = Dinv + (int64_t)ks * n;
        const int* P = A.luP + (int64_t)ks * n;
        const int64_t o = (int64_t)ch * n;
        // prologue: the input vector, in global memory
        const c2<T>* b = r + o;
        if (mode == 1) {
            c2<T> beta = from_d<T>(st->beta), omega = from_d<T>(st->omega);
            for (int i = lane; i < n; i += 32) {
                c2<T> pv = io[o + i], vv = v[o + i], rv = r[o + i];
                c2<T> t = cm<T>(omega, vv);
                c2<T> q = cm<T>(beta, mk<T>(pv.x - t.x, pv.y - t.y));
                io[o + i] = mk<T>(rv.x + q.x, rv.y + q.y);
            }
            b = io + o;
        } else if (mode == 2) {
            c2<T> alpha = from_d<T>(st->alpha);
            for (int i = lane; i < n; i += 32) {
                c2<T> t = cm<T>(alpha, v[o + i]);
                c2<T> rv = r[o + i];
                c2<T> sv = mk<T>(rv.x - t.x, rv.y - t.y);
                io[o + i] = sv;
                nsum += (double)sv.x * sv.x + (double)sv.y * sv.y;
            }
            b = io + o;
        }
        __syncwarp();   // the prologue's stores are visible to the warp's copies below
        c2<T>* zo = z + o;
        const int nc = (n + PCH - 1) / PCH;
        auto copy_vec = [&](const c2<T>* src, int c) {   // vector chunk c (rows < n) into its ring slot
            int j0 = c * PCH, rows = min(PCH, n - j0);
            if (rows > 0) warp_copy16(Vb + (c % ROT_VRING) * PCH, src + j0, rows * (int)sizeof(c2<T>), lane);
        };
        // forward group c: factor chunk c and input chunk c + 1 (input chunk 0 goes with group 0)
        auto issue_fwd = [&](int c, int bb) {
            int j0 = c * PCH, rows = min(PCH, n - j0);
            warp_copy16(Lb + bb * PCH * KB, Lk + (int64_t)j0 * KB, rows * KB * (int)sizeof(c2<T>), lane);
            for (int e = lane; e < rows; e += 32) cp_async4(Pb + bb * PCH + e, P + j0 + e);
            if (c == 0) copy_vec(b, 0);
            copy_vec(b, c + 1);
            cp_async_commit();
        };
        issue_fwd(0, 0);
        // forward: lane l holds row j + ((l - j) mod 32); rows j .. j + KB form the window
        c2<T> w = mk<T>(0, 0);
        for (int c = 0; c < nc; c++) {
            if (c + 1 < nc) {
                issue_fwd(c + 1, (c + 1) & 1);
                cp_async_wait1();
            } else {
                cp_async_wait0();
            }
            __syncwarp();
            if (c == 0 && lane < KB && lane < n) w = Vb[lane];   // rows 0 .. KB - 1 start the window
            const c2<T>* Lc = Lb + (c & 1) * PCH * KB;
            const int* Pc = Pb + (c & 1) * PCH;
            const int j0 = c * PCH, rows = min(PCH, n - j0);
#pragma unroll
            for (int jj = 0; jj < PCH; jj++) {
                if (jj >= rows) break;
                const int j = j0 + jj;
                const int k = (lane - j) & 31;   // this lane's row is j + k
                // row j + KB enters the window: its input, from chunk c or c + 1 of the ring
                const c2<T> vin = Vb[((c + (jj + KB) / PCH) % ROT_VRING) * PCH + (jj + KB) % PCH];
                if (k == KB) w = vin;
                c2<T> lcur = (k >= 1 && k <= KB) ? Lc[jj * KB + k - 1] : mk<T>(0, 0);
                const int pj = Pc[jj] - j;
                const int l0 = j & 31, lp = (j + pj) & 31;
                c2<T> zj = shfl2<T>(w, lp), w0 = shfl2<T>(w, l0);
                if (lane == lp && pj != 0) w = w0;   // recorded interchange of rows j and j + pj
                if (k >= 1 && k <= KB && j + k < n) {
                    w.x -= lcur.x * zj.x - lcur.y * zj.y;
                    w.y -= lcur.x * zj.y + lcur.y * zj.x;
                }
                if (lane == l0) zo[j] = zj;
            }
            __syncwarp();   // buffers (c & 1) and ring slot c are refilled by later copies
        }
        __syncwarp();   // the forward results are visible to the warp's copies below
        // backward group q (chunk c = nc - 1 - q): factor chunk c and forward-result chunk c
        auto issue_bwd = [&](int c, int bb) {
            int i0 = c * PCH, rows = min(PCH, n - i0);
            warp_copy16(Ub + bb * PCH * (WU + 1), Uk + (int64_t)i0 * (WU + 1), rows * (WU + 1) * (int)sizeof(c2<T>),
                        lane);
            warp_copy16(Db + bb * PCH, Dk + i0, rows * (int)sizeof(c2<T>), lane);
            copy_vec(zo, c);
            cp_async_commit();
        };
        issue_bwd(nc - 1, 0);
        // backward: lane l holds row i - m, m = (i - l) mod 32; rows i - 1 .. i - WU accumulate
        c2<T> acc = mk<T>(0, 0), x = mk<T>(0, 0);
        for (int q = 0; q < nc; q++) {
            const int c = nc - 1 - q;
            if (c > 0) {
                issue_bwd(c - 1, (q + 1) & 1);
                cp_async_wait1();
            } else {
                cp_async_wait0();
            }
            __syncwarp();
            const c2<T>* Uc = Ub + (q & 1) * PCH * (WU + 1);
            const c2<T>* Dc = Db + (q & 1) * PCH;
            const c2<T>* Zc = Vb + (c % ROT_VRING) * PCH;
            const int i0 = c * PCH, rows = min(PCH, n - i0);
#pragma unroll
            for (int iq = 0; iq < PCH; iq++) {
                const int ii = rows - 1 - iq;
                if (ii < 0) break;
                const int i = i0 + ii;
                const int m = (i - lane) & 31;
                c2<T> ucur = (m >= 1 && m <= WU && i - m >= 0) ? Uc[ii * (WU + 1) + m] : mk<T>(0, 0);
                const c2<T> zi = Zc[ii], di = Dc[ii];
                if (m == 0) x = cm<T>(mk<T>(zi.x - acc.x, zi.y - acc.y), di);
                c2<T> xi = shfl2<T>(x, i & 31);
                if (m >= 1 && m <= WU) {
                    acc.x += ucur.x * xi.x - ucur.y * xi.y;
                    acc.y += ucur.x * xi.y + ucur.y * xi.x;
                }
                if (m == 0) {
                    zo[i] = xi;
                    acc = mk<T>(0, 0);   // the lane's next row is i - 32
                }
            }
            __syncwarp();
        }
    }
    if (part_nrm) block_reduce_store(make_double2(0, 0), nsum, nullptr, part_nrm, blockIdx.x);
}

template <class T>
size_t precond_rot_smem()
{
    return (size_t)prec_rot_warps<T>() * prec_rot_warp_bytes<T, 13>();
}

template <class T>
cudaError_t precond_rot_prepare()
{
    return cudaFuncSetAttribute(k_precond_rot<T, 13>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)precond_rot_smem<T>());
}

template <class T>
int precond_rot_blocks(int nch)
{
    return (nch + prec_rot_warps<T>() - 1) / prec_rot_warps<T>();
}

template <class T>
void launch_precond_rot_t(cudaStream_t st, const OpView& A, const void* U, const void* L, const void* Dinv, int mode,
                          const KState* ks, const void* r, const void* v, void* io, void* z, double* pn)
{
    k_precond_rot<T, 13><<<precond_rot_blocks<T>(A.nch), 32 * prec_rot_warps<T>(), precond_rot_smem<T>(), st>>>(
        A, (const c2<T>*)U, (const c2<T>*)L, (const c2<T>*)Dinv, mode, ks, (const c2<T>*)r, (const c2<T>*)v,
        (c2<T>*)io, (c2<T>*)z, pn);
}
template cudaError_t precond_rot_prepare<double>();
template cudaError_t precond_rot_prepare<float>();
template int precond_rot_blocks<double>(int);
template int precond_rot_blocks<float>(int);
template void launch_precond_rot_t<double>(cudaStream_t, const OpView&, const void*, const void*, const void*, int,
                                           const KState*, const void*, const void*, void*, void*, double*);
template void launch_precond_rot_t<float>(cudaStream_t, const OpView&, const void*, const void*, const void*, int,
                                          const KState*, const void*, const void*, void*, void*, double*);

template <class T>
size_t precond_sm_smem(int n1)
{
    return (size_t)prec_sm_warps<T>() * prec_sm_warp_bytes<T, 13>(2 * n1);
}

// The dynamic shared memory limit is a property of the kernel, shared by every operator in the
// process: it is raised to the device's opt-in maximum (never lowered to one operator's need, which
// would make a larger operator's launches fail), and an operator whose need exceeds it is refused.
template <class T>
cudaError_t precond_sm_prepare(int n1)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_precond_sm<T, 13>);
    if (e != cudaSuccess) return e;
    int lim = optin - (int)fa.sharedSizeBytes;   // static shared memory counts against the same limit
    if (precond_sm_smem<T>(n1) > (size_t)lim) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_precond_sm<T, 13>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <class T>
int precond_sm_blocks(int nch)
{
    return (nch + prec_sm_warps<T>() - 1) / prec_sm_warps<T>();
}

template <class T>
void launch_precond_sm_t(cudaStream_t st, const OpView& A, const void* U, const void* L, const void* Dinv, int mode,
                         const KState* ks, const void* r, const void* v, void* io, void* z, double* pn)
{
    int wb = (int)prec_sm_warp_bytes<T, 13>(2 * A.n1);
    k_precond_sm<T, 13><<<precond_sm_blocks<T>(A.nch), 32 * prec_sm_warps<T>(), precond_sm_smem<T>(A.n1), st>>>(
        A, (const c2<T>*)U, (const c2<T>*)L, (const c2<T>*)Dinv, mode, ks, (const c2<T>*)r, (const c2<T>*)v,
        (c2<T>*)io, (c2<T>*)z, pn, wb);
}
template size_t precond_sm_smem<double>(int);
template size_t precond_sm_smem<float>(int);
template cudaError_t precond_sm_prepare<double>(int);
template cudaError_t precond_sm_prepare<float>(int);
template int precond_sm_blocks<double>(int);
template int precond_sm_blocks<float>(int);
template void launch_precond_sm_t<double>(cudaStream_t, const OpView&, const void*, const void*, const void*, int,
                                          const KState*, const void*, const void*, void*, void*, double*);
template void launch_precond_sm_t<float>(cudaStream_t, const OpView&, const void*, const void*, const void*, int,
                                         const KState*, const void*, const void*, void*, void*, double*);

// ---------------------------------------------------------------------------------------------
// x += alpha ph + omega sh;  r = s - omega t;  partials <rh, r>, ||r||^2.  After the s-check ended
// the solve (done == 2): x += alpha ph only.  A block of UXR_T threads covers 2 UXR_T elements (two
// per thread, a warp's loads contiguous), so the FP64 block reduction is paid once per two.
// ---------------------------------------------------------------------------------------------
constexpr int UXR_T = 128;

template <class T>
__global__ void __launch_bounds__(UXR_T) k_update_xr(int64_t n, const KState* st, c2<T>* x, c2<T>* r,
                                                     const c2<T>* ph, const c2<T>* sh, const c2<T>* s,
                                                     const c2<T>* t, const c2<T>* rh, double2* part_dot,
                                                     double* part_nrm)
{
    const int64_t base = (int64_t)blockIdx.x * (2 * UXR_T) + threadIdx.x;
    double2 dsum = make_double2(0, 0);
    double nsum = 0;
    if (st->status == 0 && st->done != 1) {
        const c2<T> al = from_d<T>(st->alpha), om = from_d<T>(st->omega);
        const bool only_x = st->done == 2;
        for (int k = 0; k < 2; k++) {
            const int64_t i = base + k * UXR_T;
            if (i >= n) break;
            c2<T> a = cm<T>(al, ph[i]);
            if (only_x) {
                x[i].x += a.x;
                x[i].y += a.y;
                continue;
            }
            c2<T> w = cm<T>(om, sh[i]);
            x[i].x += a.x + w.x;
            x[i].y += a.y + w.y;
            c2<T> ot = cm<T>(om, t[i]);
            c2<T> rn = mk<T>(s[i].x - ot.x, s[i].y - ot.y);
            r[i] = rn;
            c2<T> h = rh[i];
            dsum.x += (double)h.x * rn.x + (double)h.y * rn.y;
            dsum.y += (double)h.x * rn.y - (double)h.y * rn.x;
            nsum += (double)rn.x * rn.x + (double)rn.y * rn.y;
        }
    }
    block_reduce_store(dsum, nsum, part_dot, part_nrm, blockIdx.x);
}

// blocks = the partial slots of the vector kernels: one per 256 elements
template <class T>
void launch_update_xr_t(int blocks, cudaStream_t st, int64_t n, const KState* ks, void* x, void* r, const void* ph,
                        const void* sh, const void* s, const void* t, const void* rh, double2* pd, double* pn)
{
    static_assert(2 * UXR_T == 256, "one block per 256 elements, as the other vector kernels");
    k_update_xr<T><<<blocks, UXR_T, 0, st>>>(n, ks, (c2<T>*)x, (c2<T>*)r, (const c2<T>*)ph, (const c2<T>*)sh,
                                             (const c2<T>*)s, (const c2<T>*)t, (const c2<T>*)rh, pd, pn);
}
template void launch_update_xr_t<double>(int, cudaStream_t, int64_t, const KState*, void*, void*, const void*,
                                         const void*, const void*, const void*, const void*, double2*, double*);
template void launch_update_xr_t<float>(int, cudaStream_t, int64_t, const KState*, void*, void*, const void*,
                                        const void*, const void*, const void*, const void*, double2*, double*);

// ---------------------------------------------------------------------------------------------
// Precision conversions of the refinement loop: d32 = r64 / ||r|| (scaled inner right-hand side)
// and x64 += ||r|| d32.  The outer KState's rnorm2 holds ||r||^2.  The scale is formed once per
// block: an FP64 square root and division per element would make these copies FP64-bound.
// ---------------------------------------------------------------------------------------------
__global__ void k_to_float_scaled(int64_t n, const double2* a, const KState* st, float2* b)
{
    __shared__ double sc;
    if (threadIdx.x == 0) sc = st->rnorm2 > 0 ? 1.0 / sqrt(st->rnorm2) : 0.0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = sc;
    const double2 v = a[i];
    b[i] = make_float2((float)(v.x * s), (float)(v.y * s));
}

__global__ void k_add_float_scaled(int64_t n, const float2* d, const KState* st, double2* x)
{
    __shared__ double sc;
    if (threadIdx.x == 0) sc = sqrt(st->rnorm2);
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = sc;
    const float2 dv = d[i];
    double2 xv = x[i];
    xv.x += s * (double)dv.x;
    xv.y += s * (double)dv.y;
    x[i] = xv;
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
