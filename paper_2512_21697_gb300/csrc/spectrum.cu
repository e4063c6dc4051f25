// spectrum.cu -- differential photoelectron energy spectrum (Sec. 4.3, Eq. dPdE):
//   dP/dE = sum over the channels (kappa, mu) of |<psi_{kappa mu E} | Psi>|^2.
//
// The continuum states of a kappa are its eigenvectors v_j of H0_kappa v = E S_kappa v in the
// energy window (e_lo, e_hi] (normalised v^T S v = 1, the box's discrete continuum).  Dividing a
// box-normalised state by the square root of the local level spacing dE_j (the central difference
// of the neighbouring levels, one-sided at the window's two ends) makes it energy-normalised, so
// at the levels dP/dE_kappa(E_j) = sum over mu of |v_j^T S_kappa Psi_{kappa mu}|^2 / dE_j.  The
// spectrum on a user grid is the linear interpolation of each kappa's densities in E (zero outside
// its first and last level in the window; a kappa with fewer than two levels there adds nothing),
// summed over kappa in ascending slot order.
//
// The eigenpairs depend on kappa and the window only: computed once per window (cuSOLVER, see
// eig_window) and kept on the device.  Three kernels per call:
//   k_spec_proj     block per channel: S Psi_ch in shared memory, a warp per eigenvector forms the
//                   projection (fixed shuffle tree) and stores |.|^2;
//   k_spec_density  thread per level: the sum over the kappa's channels (ascending) / dE_j;
//   k_spec_grid     thread per grid point: the interpolated densities summed over kappa.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "device.h"
#include "internal.h"
#include "kernels.h"
#include "op.h"

namespace dg {

struct SpecState {
    double e_lo = 0, e_hi = 0;
    bool valid = false;
    int nk2 = 0, nvec = 0;
    double* vec = nullptr;      // [vector][2 n1], slot order
    double* E = nullptr;        // [vector], ascending within a kappa slot
    int* vstart = nullptr;      // first vector of each kappa slot [nk2 + 1]
    int* vslot = nullptr;       // kappa slot of each vector
    int64_t nq = 0;
    double* q = nullptr;        // |v^T S psi_ch|^2 per (channel, vector of its kappa slot)
    int64_t* choff = nullptr;   // first entry of each channel in q
    int* kch_start = nullptr;   // channels of each kappa slot, ascending: kch[kch_start[ks] ..]
    int* kch = nullptr;
    double* dens = nullptr;     // per vector: density at the level
    double* grid = nullptr;     // device copies of the user grid and the result
    double* P = nullptr;
    int grid_cap = 0;
};

namespace {

void spec_release(SpecState* s)
{
    void* ptrs[] = {s->vec, s->E, s->vstart, s->vslot, s->q, s->choff, s->kch_start, s->kch, s->dens};
    for (void* p : ptrs) cudaFree(p);
    s->vec = s->E = s->q = s->dens = nullptr;
    s->vstart = s->vslot = s->kch_start = s->kch = nullptr;
    s->choff = nullptr;
    s->valid = false;
    s->nvec = 0;
    s->nq = 0;
}

__global__ void k_spec_proj(OpView A, const double2* __restrict__ psi, const double* __restrict__ vec,
                            const int* __restrict__ vstart, const int64_t* __restrict__ choff,
                            double* __restrict__ q)
{
    extern __shared__ double2 sx[];   // S psi of this channel, 2 n1 entries
    const int ch = blockIdx.x, ks = A.ch_kslot[ch], n1 = A.n1, ns = 2 * n1;
    const double2* xa = psi + (int64_t)ch * ns;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        const int r = i >> 1, t = i & 1;
        const double* Sk = A.S + ((int64_t)ks * n1 + r) * A.bd * 4;
        double2 acc = make_double2(0, 0);
        for (int d = 0; d < A.bd; d++) {
            const int rr = r + d - A.half;
            if (rr < 0 || rr >= n1) continue;
            for (int u = 0; u < 2; u++) {
                const double s = Sk[d * 4 + t * 2 + u];
                const double2 x = xa[2 * rr + u];
                acc.x += s * x.x;
                acc.y += s * x.y;
            }
        }
        sx[i] = acc;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int v0 = vstart[ks], v1 = vstart[ks + 1];
    double* qc = q + choff[ch];
    for (int v = v0 + warp; v < v1; v += nw) {
        const double* w = vec + (int64_t)v * ns;
        double2 pr = make_double2(0, 0);
        for (int i = lane; i < ns; i += 32) {
            const double wi = w[i];
            pr.x += wi * sx[i].x;
            pr.y += wi * sx[i].y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            pr.x += __shfl_down_sync(0xffffffffu, pr.x, o);
            pr.y += __shfl_down_sync(0xffffffffu, pr.y, o);
        }
        if (lane == 0) qc[v - v0] = pr.x * pr.x + pr.y * pr.y;
    }
}

__global__ void k_spec_density(int nvec, const double* __restrict__ E, const int* __restrict__ vstart,
                               const int* __restrict__ vslot, const int64_t* __restrict__ choff,
                               const int* __restrict__ kch_start, const int* __restrict__ kch,
                               const double* __restrict__ q, double* __restrict__ dens)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvec) return;
    const int ks = vslot[v], v0 = vstart[ks], m = vstart[ks + 1] - v0, j = v - v0;
    if (m < 2) {
        dens[v] = 0.0;
        return;
    }
    double sum = 0.0;
    for (int c = kch_start[ks]; c < kch_start[ks + 1]; c++) sum += q[choff[kch[c]] + j];
    const double* Ek = E + v0;
    const double dE = j == 0 ? Ek[1] - Ek[0] : j == m - 1 ? Ek[m - 1] - Ek[m - 2] : 0.5 * (Ek[j + 1] - Ek[j - 1]);
    dens[v] = sum / dE;
}

__global__ void k_spec_grid(int ngrid, const double* __restrict__ grid, int nk2, const double* __restrict__ E,
                            const int* __restrict__ vstart, const double* __restrict__ dens, double* __restrict__ P)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngrid) return;
    const double x = grid[g];
    double acc = 0.0;
    for (int ks = 0; ks < nk2; ks++) {
        const int v0 = vstart[ks], m = vstart[ks + 1] - v0;
        if (m < 2) continue;
        const double* Ek = E + v0;
        const double* dk = dens + v0;
        if (!(x >= Ek[0] && x <= Ek[m - 1])) continue;
        // the last level j with Ek[j] <= x (binary search over ascending levels)
        int lo = 0, hi = m - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (Ek[mid] <= x) lo = mid;
            else hi = mid - 1;
        }
        if (lo == m - 1) {
            acc += dk[m - 1];
        } else {
            const double w = (x - Ek[lo]) / (Ek[lo + 1] - Ek[lo]);
            acc += dk[lo] + w * (dk[lo + 1] - dk[lo]);
        }
    }
    P[g] = acc;
}

#define SPTRY(call)                                                                                \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            set_error(std::string("dirac_spectrum: ") + #call + ": " + cudaGetErrorString(e_));    \
            return DIRAC_E_CUDA;                                                                   \
        }                                                                                          \
    } while (0)

template <typename T>
cudaError_t put(T** d, const std::vector<T>& h, cudaStream_t st)
{
    cudaError_t e = cudaMalloc(d, sizeof(T) * std::max<size_t>(h.size(), 1));
    if (e == cudaSuccess && !h.empty()) e = cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st);
    return e;
}

// eigenpairs of the window and the index tables, once per window
dirac_status spec_setup(dirac_op* op, double e_lo, double e_hi)
{
    if (!op->spec) op->spec = new SpecState();
    SpecState* s = op->spec;
    if (s->valid && s->e_lo == e_lo && s->e_hi == e_hi) return DIRAC_OK;
    SPTRY(cudaStreamSynchronize(op->st));
    spec_release(s);
    const Basis& B = op->B;
    const int nk2 = 2 * B.p.kappa_max;
    std::vector<double> hvec, hE;
    std::vector<int> hstart;
    dirac_status e = eig_window(op, e_lo, e_hi, hvec, hE, hstart);
    if (e) return e;
    const int nvec = hstart[nk2];
    std::vector<int> vslot(nvec);
    for (int ks = 0; ks < nk2; ks++)
        for (int v = hstart[ks]; v < hstart[ks + 1]; v++) vslot[v] = ks;
    std::vector<int64_t> choff(B.nch + 1, 0);
    for (int ch = 0; ch < B.nch; ch++) {
        const int ks = kappa_slot(B.kap[ch]);
        choff[ch + 1] = choff[ch] + (hstart[ks + 1] - hstart[ks]);
    }
    std::vector<int> kcs(nk2 + 1, 0), kc;
    for (int ks = 0; ks < nk2; ks++) {
        for (int ch = 0; ch < B.nch; ch++)
            if (kappa_slot(B.kap[ch]) == ks) kc.push_back(ch);
        kcs[ks + 1] = (int)kc.size();
    }
    SPTRY(put(&s->vec, hvec, op->st));
    SPTRY(put(&s->E, hE, op->st));
    SPTRY(put(&s->vstart, hstart, op->st));
    SPTRY(put(&s->vslot, vslot, op->st));
    SPTRY(put(&s->choff, choff, op->st));
    SPTRY(put(&s->kch_start, kcs, op->st));
    SPTRY(put(&s->kch, kc, op->st));
    SPTRY(cudaMalloc(&s->q, sizeof(double) * std::max<int64_t>(choff[B.nch], 1)));
    SPTRY(cudaMalloc(&s->dens, sizeof(double) * std::max(nvec, 1)));
    SPTRY(cudaStreamSynchronize(op->st));
    s->nk2 = nk2;
    s->nvec = nvec;
    s->nq = choff[B.nch];
    s->e_lo = e_lo;
    s->e_hi = e_hi;
    s->valid = true;
    return DIRAC_OK;
}

}  // namespace

void spec_free(dirac_op* op)
{
    if (!op->spec) return;
    spec_release(op->spec);
    cudaFree(op->spec->grid);
    cudaFree(op->spec->P);
    delete op->spec;
    op->spec = nullptr;
}

}  // namespace dg

using namespace dg;

extern "C" dirac_status dirac_spectrum(dirac_op* op, const void* psi_dev, double e_lo, double e_hi, int n_grid,
                                       const double* e_grid, double* dpde, int64_t* counts)
{
    if (!op || !psi_dev || !std::isfinite(e_lo) || !std::isfinite(e_hi) || !(e_lo < e_hi) || n_grid < 0 ||
        n_grid > (1 << 26) || (n_grid > 0 && (!e_grid || !dpde))) {
        set_error("dirac_spectrum: bad argument");
        return DIRAC_E_ARG;
    }
    for (int g = 0; g < n_grid; g++)
        if (!std::isfinite(e_grid[g])) {
            set_error("dirac_spectrum: non-finite grid energy");
            return DIRAC_E_ARG;
        }
    dirac_status e = spec_setup(op, e_lo, e_hi);
    if (e) return e;
    SpecState* s = op->spec;
    const int ns = 2 * op->ov.n1;
    const size_t smem = sizeof(double2) * ns;
    if (smem > 48 * 1024) {
        int dev = 0, optin = 0;
        SPTRY(cudaGetDevice(&dev));
        SPTRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (smem > (size_t)optin) {
            set_error("dirac_spectrum: radial size too large for the projection kernel");
            return DIRAC_E_ARG;
        }
        SPTRY(cudaFuncSetAttribute(k_spec_proj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (n_grid > s->grid_cap) {
        cudaFree(s->grid);
        cudaFree(s->P);
        s->grid = s->P = nullptr;
        s->grid_cap = 0;
        SPTRY(cudaMalloc(&s->grid, sizeof(double) * n_grid));
        SPTRY(cudaMalloc(&s->P, sizeof(double) * n_grid));
        s->grid_cap = n_grid;
    }
    if (s->nvec > 0) {
        k_spec_proj<<<op->ov.nch, 256, smem, op->st>>>(op->ov, (const double2*)psi_dev, s->vec, s->vstart, s->choff,
                                                       s->q);
        k_spec_density<<<grid_for(s->nvec, 256), 256, 0, op->st>>>(s->nvec, s->E, s->vstart, s->vslot, s->choff,
                                                                   s->kch_start, s->kch, s->q, s->dens);
        op->launches += 2;
    }
    if (n_grid > 0) {
        SPTRY(cudaMemcpyAsync(s->grid, e_grid, sizeof(double) * n_grid, cudaMemcpyHostToDevice, op->st));
        k_spec_grid<<<grid_for(n_grid, 128), 128, 0, op->st>>>(n_grid, s->grid, s->nvec > 0 ? s->nk2 : 0, s->E,
                                                               s->vstart, s->dens, s->P);
        op->launches++;
        SPTRY(cudaGetLastError());
        SPTRY(cudaMemcpyAsync(dpde, s->P, sizeof(double) * n_grid, cudaMemcpyDeviceToHost, op->st));
    }
    SPTRY(cudaGetLastError());
    SPTRY(cudaStreamSynchronize(op->st));
    if (counts) {
        counts[0] = s->nvec;
        counts[1] = s->nq;
    }
    return DIRAC_OK;
}

extern "C" dirac_status dirac_spectrum_error(int n_grid, const double* e_grid, const double* p_n, const double* p_m,
                                             double e1, double e2, double* err)
{
    if (n_grid < 0 || (n_grid > 0 && (!e_grid || !p_n || !p_m)) || !err || !(e1 <= e2)) {
        set_error("dirac_spectrum_error: bad argument");
        return DIRAC_E_ARG;
    }
    double acc = 0.0, pe = 0.0, pf = 0.0;
    bool have = false;
    for (int g = 0; g < n_grid; g++) {
        if (g > 0 && !(e_grid[g] > e_grid[g - 1])) {
            set_error("dirac_spectrum_error: the grid must ascend");
            return DIRAC_E_ARG;
        }
        if (!(e_grid[g] >= e1 && e_grid[g] <= e2)) continue;
        const double d = p_n[g] - p_m[g], f = d * d;
        if (have) acc += 0.5 * (f + pf) * (e_grid[g] - pe);
        pe = e_grid[g];
        pf = f;
        have = true;
    }
    *err = acc;
    return DIRAC_OK;
}
