// bound.cu -- population of the bound states (Sec. 4.3): P_bound = sum over the channels (kappa, mu)
// and over the bound eigenvectors v_b of H0_kappa v = E S_kappa v with -c^2 < E < 0 (the
// positive-energy bound branch in the shifted-energy convention) of |v_b^T S_kappa psi_{kappa mu}|^2.
//
// The eigenvectors depend on kappa only.  They are computed once per operator, on the first request,
// by cuSOLVER's dense generalised symmetric-definite eigensolver restricted to the eigenvalue window
// (-c^2, 0] (one call per kappa, on the functions that kappa uses, normalised v^T S v = 1), and kept
// on the device expanded to the library's slot order.  The projection is one kernel: a block per
// channel forms S psi in shared memory and reduces every bound vector against it.
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <string>
#include <vector>

#include "device.h"
#include "internal.h"
#include "kernels.h"
#include "op.h"

namespace dg {

// deterministic block sum of a double2 (fixed shuffle tree, then fixed order over the warps)
__device__ double2 block_sum2(double2 v, double2* red)
{
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0) red[w] = v;
    __syncthreads();
    double2 s = make_double2(0, 0);
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; i++) { s.x += red[i].x; s.y += red[i].y; }
    __syncthreads();
    return s;   // valid in thread 0
}

// part[ch] = sum_b |v_b^T S_kappa psi_ch|^2 over the bound vectors of the channel's kappa
__global__ void k_pbound(OpView A, const double2* __restrict__ psi, const double* __restrict__ bvec,
                         const int* __restrict__ bstart, double* __restrict__ part)
{
    extern __shared__ double2 sx[];   // S psi of this channel, 2 n1 entries
    __shared__ double2 red[32];
    int ch = blockIdx.x, ks = A.ch_kslot[ch], n1 = A.n1, ns = 2 * n1;
    const double2* xa = psi + (int64_t)ch * ns;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        int r = i >> 1, t = i & 1;
        const double* Sk = A.S + ((int64_t)ks * n1 + r) * A.bd * 4;
        double2 acc = make_double2(0, 0);
        for (int d = 0; d < A.bd; d++) {
            int rr = r + d - A.half;
            if (rr < 0 || rr >= n1) continue;
            for (int u = 0; u < 2; u++) {
                double s = Sk[d * 4 + t * 2 + u];
                double2 x = xa[2 * rr + u];
                acc.x += s * x.x;
                acc.y += s * x.y;
            }
        }
        sx[i] = acc;
    }
    __syncthreads();
    double tot = 0;
    for (int b = bstart[ks]; b < bstart[ks + 1]; b++) {
        const double* v = bvec + (int64_t)b * ns;
        double2 pr = make_double2(0, 0);
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            double vi = v[i];
            pr.x += vi * sx[i].x;
            pr.y += vi * sx[i].y;
        }
        pr = block_sum2(pr, red);
        if (threadIdx.x == 0) tot += pr.x * pr.x + pr.y * pr.y;
    }
    if (threadIdx.x == 0) part[ch] = tot;
}

#define BTRY(call)                                                                                 \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            set_error(std::string("eigenpairs: ") + #call + ": " + cudaGetErrorString(e_));         \
            ok = DIRAC_E_CUDA;                                                                     \
            goto done;                                                                             \
        }                                                                                          \
    } while (0)
#define STRY(call)                                                                                 \
    do {                                                                                           \
        cusolverStatus_t s_ = (call);                                                              \
        if (s_ != CUSOLVER_STATUS_SUCCESS) {                                                       \
            set_error(std::string("eigenpairs: ") + #call + " failed with status " +               \
                      std::to_string((int)s_));                                                    \
            ok = DIRAC_E_NUMERIC;                                                                  \
            goto done;                                                                             \
        }                                                                                          \
    } while (0)

// Eigenpairs of H0_kappa v = E S_kappa v with vl < E <= vu for every kappa slot in use: cuSOLVER's
// dense generalised symmetric-definite solver restricted to the window, on the functions the kappa
// uses (v^T S v = 1), the vectors expanded to the library's slot order.  Host results: hvec
// [vector][2 n1], hE [vector] (ascending within a slot), hstart [2 kappa_max + 1].
dirac_status eig_window(dirac_op* op, double vl, double vu, std::vector<double>& hvec, std::vector<double>& hE,
                        std::vector<int>& hstart)
{
    const Basis& B = op->B;
    int n1 = B.n1, ns = 2 * n1, nk2 = 2 * B.p.kappa_max;
    std::vector<int> used(nk2, 0);
    for (int ch = 0; ch < B.nch; ch++) used[kappa_slot(B.kap[ch])] = 1;
    hstart.assign(nk2 + 1, 0);
    hvec.clear();
    hE.clear();
    dirac_status ok = DIRAC_OK;
    cusolverDnHandle_t h = nullptr;
    double *dA = nullptr, *dB = nullptr, *dW = nullptr, *work = nullptr;
    int* dinfo = nullptr;
    int lwork_cap = 0;
    std::vector<double> hA, hB, hV;
    STRY(cusolverDnCreate(&h));
    STRY(cusolverDnSetStream(h, op->st));
    BTRY(cudaMalloc(&dA, sizeof(double) * ns * ns));
    BTRY(cudaMalloc(&dB, sizeof(double) * ns * ns));
    BTRY(cudaMalloc(&dW, sizeof(double) * ns));
    BTRY(cudaMalloc(&dinfo, sizeof(int)));
    for (int ks = 0; ks < nk2; ks++) {
        hstart[ks + 1] = hstart[ks];
        if (!used[ks]) continue;
        int kappa = (ks % 2 ? 1 : -1) * (ks / 2 + 1);
        Band S, H;
        radial_blocks(B, kappa, S, H);
        std::vector<int> act;
        for (int i = 0; i < ns; i++)
            if (slot_used(kappa, i / 2, i % 2)) act.push_back(i);
        int m = (int)act.size();
        hA.assign((size_t)m * m, 0.0);
        hB.assign((size_t)m * m, 0.0);
        for (int j = 0; j < m; j++)
            for (int i = 0; i < m; i++) {   // column major; the band keeps this cheap to fill
                if (std::abs(act[i] / 2 - act[j] / 2) > B.half) continue;
                hA[(size_t)j * m + i] = band_entry(H, act[i], act[j]);
                hB[(size_t)j * m + i] = band_entry(S, act[i], act[j]);
            }
        BTRY(cudaMemcpyAsync(dA, hA.data(), sizeof(double) * m * m, cudaMemcpyHostToDevice, op->st));
        BTRY(cudaMemcpyAsync(dB, hB.data(), sizeof(double) * m * m, cudaMemcpyHostToDevice, op->st));
        int meig = 0, lwork = 0;
        STRY(cusolverDnDsygvdx_bufferSize(h, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_V,
                                          CUBLAS_FILL_MODE_LOWER, m, dA, m, dB, m, vl, vu, 0, 0, &meig, dW,
                                          &lwork));
        if (lwork > lwork_cap) {
            if (work) cudaFree(work);
            work = nullptr;
            BTRY(cudaMalloc(&work, sizeof(double) * (size_t)lwork));
            lwork_cap = lwork;
        }
        STRY(cusolverDnDsygvdx(h, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_V,
                               CUBLAS_FILL_MODE_LOWER, m, dA, m, dB, m, vl, vu, 0, 0, &meig, dW, work, lwork,
                               dinfo));
        int info = 0;
        std::vector<double> Ew(std::max(meig, 1));
        BTRY(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, op->st));
        if (meig > 0) {
            hV.resize((size_t)m * meig);
            BTRY(cudaMemcpyAsync(hV.data(), dA, sizeof(double) * m * meig, cudaMemcpyDeviceToHost, op->st));
            BTRY(cudaMemcpyAsync(Ew.data(), dW, sizeof(double) * meig, cudaMemcpyDeviceToHost, op->st));
        }
        BTRY(cudaStreamSynchronize(op->st));
        if (info != 0) {
            set_error("eigenpairs: generalised eigensolver info " + std::to_string(info) + " for kappa " +
                      std::to_string(kappa));
            ok = DIRAC_E_NUMERIC;
            goto done;
        }
        for (int e = 0; e < meig; e++) {
            if (!(Ew[e] > vl && Ew[e] <= vu)) continue;
            size_t o = hvec.size();
            hvec.resize(o + ns, 0.0);
            for (int i = 0; i < m; i++) hvec[o + act[i]] = hV[(size_t)e * m + i];
            hE.push_back(Ew[e]);
            hstart[ks + 1]++;
        }
    }
done:
    if (h) cusolverDnDestroy(h);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dW);
    cudaFree(work);
    cudaFree(dinfo);
    return ok;
}

// Bound eigenvectors of every kappa in use (-c^2 < E < 0), into op->bvec / op->bstart (device), once.
dirac_status bound_setup(dirac_op* op)
{
    if (op->bvec) return DIRAC_OK;
    const Basis& B = op->B;
    int nk2 = 2 * B.p.kappa_max, ns = 2 * B.n1;
    double c2 = B.p.c * B.p.c;
    std::vector<double> wvec, wE;
    std::vector<int> wstart;
    dirac_status ok = eig_window(op, -c2, 0.0, wvec, wE, wstart);
    if (ok) return ok;
    std::vector<int> hstart(nk2 + 1, 0);
    std::vector<double> hvec;
    for (int ks = 0; ks < nk2; ks++) {
        hstart[ks + 1] = hstart[ks];
        for (int v = wstart[ks]; v < wstart[ks + 1]; v++) {
            if (!(wE[v] < 0)) continue;
            hvec.insert(hvec.end(), wvec.begin() + (size_t)v * ns, wvec.begin() + (size_t)(v + 1) * ns);
            hstart[ks + 1]++;
        }
    }
    {
        int nvec = hstart[nk2];
        double* dv = nullptr;
        int* dst = nullptr;
        double* dp = nullptr;
        BTRY(cudaMalloc(&dv, sizeof(double) * std::max<size_t>(hvec.size(), 1)));
        op->allocs.push_back(dv);
        BTRY(cudaMalloc(&dst, sizeof(int) * (nk2 + 1)));
        op->allocs.push_back(dst);
        BTRY(cudaMalloc(&dp, sizeof(double) * B.nch));
        op->allocs.push_back(dp);
        if (!hvec.empty())
            BTRY(cudaMemcpyAsync(dv, hvec.data(), sizeof(double) * hvec.size(), cudaMemcpyHostToDevice, op->st));
        BTRY(cudaMemcpyAsync(dst, hstart.data(), sizeof(int) * (nk2 + 1), cudaMemcpyHostToDevice, op->st));
        BTRY(cudaStreamSynchronize(op->st));
        op->bytes += sizeof(double) * hvec.size();
        op->bvec = dv;
        op->bstart = dst;
        op->part_pb = dp;
        op->nbound = nvec;
    }
done:
    return ok;
}

// P_bound of psi (synchronises the op's stream)
dirac_status bound_population(dirac_op* op, const double2* psi, double* out)
{
    dirac_status e = bound_setup(op);
    if (e) return e;
    int ns = 2 * op->ov.n1;
    size_t smem = sizeof(double2) * ns;
    if (smem > 48 * 1024) {
        // the limit is per kernel and shared by every operator: raise it to the device maximum
        int dev = 0, optin = 0;
        cudaError_t ce = cudaGetDevice(&dev);
        if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        if (ce == cudaSuccess) ce = cudaFuncGetAttributes(&fa, k_pbound);
        int lim = ce == cudaSuccess ? optin - (int)fa.sharedSizeBytes : 0;   // static shared memory included
        if (ce == cudaSuccess && smem <= (size_t)lim)
            ce = cudaFuncSetAttribute(k_pbound, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (ce != cudaSuccess || smem > (size_t)lim) {
            set_error("bound states: radial size too large for the projection kernel");
            return DIRAC_E_ARG;
        }
    }
    k_pbound<<<op->ov.nch, 256, smem, op->st>>>(op->ov, psi, op->bvec, op->bstart, op->part_pb);
    op->launches++;
    e = check_launch("bound states");
    if (e) return e;
    std::vector<double> p(op->ov.nch);
    cudaError_t ce = cudaMemcpyAsync(p.data(), op->part_pb, sizeof(double) * p.size(), cudaMemcpyDeviceToHost, op->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(op->st);
    if (ce != cudaSuccess) { set_error(std::string("bound states: ") + cudaGetErrorString(ce)); return DIRAC_E_CUDA; }
    double s = 0;
    for (double v : p) s += v;
    *out = s;
    return DIRAC_OK;
}

}  // namespace dg
