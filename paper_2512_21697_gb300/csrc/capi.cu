// capi.cu -- C ABI of libdirac_gb300: operator upload, operator apply, preconditioner apply,
// the Crank-Nicolson step loop (Eq. solPsi) solved by right-preconditioned BiCGSTAB in double
// precision or by complex64 BiCGSTAB inside double-precision iterative refinement, phase timers
// and observables.  All device work is ordered on the stream given at setup.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <map>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "device.h"
#include "internal.h"
#include "kernels.h"
#include "op.h"

namespace dg {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

#define CUDA_TRY(call)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                       \
            return e_ == cudaErrorMemoryAllocation ? DIRAC_E_NOMEM : DIRAC_E_CUDA;               \
        }                                                                                        \
    } while (0)

}  // namespace dg


namespace dg {

template <class T>
static dirac_status dev_alloc(dirac_op* op, T** out, size_t count)
{
    void* p = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        set_error("cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? DIRAC_E_NOMEM : DIRAC_E_CUDA;
    }
    op->allocs.push_back(p);
    op->bytes += bytes;
    *out = (T*)p;
    return DIRAC_OK;
}

template <class T>
static dirac_status upload(dirac_op* op, T** out, const std::vector<T>& host)
{
    dirac_status s = dev_alloc(op, out, host.size());
    if (s) return s;
    if (!host.empty()) CUDA_TRY(cudaMemcpy(*out, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice));
    return DIRAC_OK;
}

int grid_for(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

// ---- phase timers: one event pair around each timed launch group, read at the next sync ----
static cudaEvent_t take_event(dirac_op* op)
{
    if (!op->event_pool.empty()) {
        cudaEvent_t e = op->event_pool.back();
        op->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

struct PhaseScope {
    dirac_op* op;
    int phase;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    PhaseScope(dirac_op* o, int ph, int nlaunch, cudaStream_t stream = nullptr)
        : op(o), phase(ph), st(stream ? stream : o->st)
    {
        op->launches += nlaunch;
        if (op->profiling) {
            a = take_event(op);
            cudaEventRecord(a, st);
        }
    }
    ~PhaseScope()
    {
        if (!a) return;
        cudaEvent_t b = take_event(op);
        cudaEventRecord(b, st);
        op->pending.push_back({phase, {a, b}});
    }
};

void collect_phases(dirac_op* op)
{
    // timers on the overlapped assembly stream may still be running: keep those for a later call
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> keep;
    for (auto& pe : op->pending) {
        if (cudaEventQuery(pe.second.second) == cudaErrorNotReady) {
            keep.push_back(pe);
            continue;
        }
        float ms = 0;
        if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
            op->phase_ms[pe.first] += ms;
            op->phase_n[pe.first] += 1;
        }
        op->event_pool.push_back(pe.second.first);
        op->event_pool.push_back(pe.second.second);
    }
    // a not-ready query is not an error of the stream; clear it only if it is what is pending
    if (!keep.empty() && cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
    op->pending.swap(keep);
}

// ---- launch helpers ------------------------------------------------------------------------
int apply_parts(const dirac_op* op, const Krylov& K)
{
    if (K.prec == 1 && op->fact32 == 1) return grid_for(op->ov.n1, FTR) * op->nfsub;
    if (K.prec == 1 && op->fact32 == 2) return grid_for(op->ov.n1, FTR) * op->ov.nch;
    return (K.prec == 1 && op->part_own) ? op->nparts_own : op->nparts_apply;
}

void k_apply_launch(dirac_op* op, const Krylov& K, int sign, const void* x, void* y, const void* bsub,
                           const void* dv, double2* pdot, double* pnrm, const KState* skip)
{
    PhaseScope ps(op, K.prec == 0 ? DIRAC_PHASE_APPLY : DIRAC_PHASE_APPLY32, 1);
    dim3 grid(op->ov.nch, grid_for(op->ov.n1, 128));
    if (K.prec == 0)
        launch_apply_t<double>(grid, op->st, op->ov, (const double*)K.S, (const double*)K.H, sign, x,
                               (const double*)K.W, y, bsub, dv, pdot, pnrm, skip);
    else if (op->fact32 == 1)
        launch_fact32_sub(op->st, op->ov, op->rad_lanes, op->nrad_lanes, op->fsub, op->nfsub, op->fsub_max,
                          op->fitem_off, op->fitem_coef, op->Ghi, op->pv.L, op->S32T, op->H32T, sign, x, op->Zf, y, bsub, dv,
                          pdot, pnrm, skip);
    else if (op->fact32 == 2)
        launch_fact32_chan(op->st, op->ov, op->rad_chunks, op->nrad, op->Gdf, op->pv.L, (const float*)K.S,
                           (const float*)K.H, sign, x, op->Zf, op->cab_df, y, bsub, dv, pdot, pnrm, skip);
    else if (op->part_own)
        launch_apply_own32(op->st, op->ov, op->S32T, op->H32T, sign, x, (const float*)K.W, y,
                           op->part_own, bsub, dv, pdot, pnrm, skip, op->dev_err);
    else
        launch_apply_t<float>(grid, op->st, op->ov, (const float*)K.S, (const float*)K.H, sign, x,
                              (const float*)K.W, y, bsub, dv, pdot, pnrm, skip);
}

// precision 2: pulse factors, combined bands and double-float coupling values of one buffer set,
// on stream st (the op's stream, or the overlap stream)
void launch_assemble_set(dirac_op* op, cudaStream_t st, const AsmSet& a)
{
    PhaseScope ps(op, DIRAC_PHASE_ASSEMBLE, op->npairs ? 4 : 2, st);
    k_time_factors<<<1, 128, 0, st>>>(op->pv, a.t_eval, a.s);
    int be = op->ov.n1 * op->ov.bd * 4;
    k_field_combine_df<<<dim3(grid_for(be, 256), op->pv.L * 4), 256, 0, st>>>(op->pv, be, a.s, a.Gdf, a.Ghi);
    if (op->npairs) {
        if (op->asm_chunks) {
            launch_assemble_grp_df(st, op->ov, op->asm_chunks, op->asm_nchunks, op->asm_gpair, op->asm_gcoef,
                                   a.Gdf, a.Wh, a.Wl);
        } else {
            k_build_K_df<<<dim3(grid_for(be, 256), (unsigned)std::min(op->ov.nkeys, 65535)), 256, 0, st>>>(
                op->ov, be, a.Gdf, a.Kdf, a.KTdf);
            launch_assemble_df(dim3(grid_for((int64_t)op->ov.n1 * op->ov.bd, 128),
                                    (unsigned)std::min<int64_t>(op->npairs, 65535)),
                               st, op->ov, a.Kdf, a.KTdf, op->cab_df, a.Wh, a.Wl);
        }
    }
}

void launch_assemble(dirac_op* op)
{
    if (op->opts.precision == 2) {
        launch_assemble_set(op, op->st, op->aset[op->acur]);
        return;
    }
    PhaseScope ps(op, DIRAC_PHASE_ASSEMBLE, op->npairs ? 4 : 2);
    k_time_factors<<<1, 128, 0, op->st>>>(op->pv, op->t_eval, op->s);
    int be = op->ov.n1 * op->ov.bd * 4;
    k_field_combine<<<dim3(grid_for(be, 256), op->pv.L * 4), 256, 0, op->st>>>(op->pv, be, op->s, op->G);
    if (op->npairs) {
        k_build_K<<<dim3(grid_for(be, 256), (unsigned)std::min(op->ov.nkeys, 65535)), 256, 0, op->st>>>(
            op->ov, be, op->G, op->K);
        k_assemble64<<<dim3(grid_for((int64_t)op->ov.n1 * op->ov.bd, 128),
                            (unsigned)std::min<int64_t>(op->npairs, 65535)), 128, 0, op->st>>>(op->ov, op->K, op->W,
                                                                                               op->W32);
    }
}

// y = A_sign x accurate to double precision (x, y, bsub complex128): native FP64 kernels, or the
// double-float kernels in precision 2
void apply_accurate(dirac_op* op, int sign, const void* x, void* y, const void* bsub, double* pnrm)
{
    if (op->opts.precision != 2) {
        k_apply_launch(op, op->k64, sign, x, y, bsub, nullptr, nullptr, pnrm, nullptr);
        return;
    }
    PhaseScope ps(op, DIRAC_PHASE_APPLY, 2);
    k_split_vec<<<op->nparts_vec, 256, 0, op->st>>>(op->n, (const double2*)x, op->xsplit);
    dim3 grid(op->ov.nch, grid_for(op->ov.n1, 128));
    launch_apply_df(grid, op->st, op->ov, op->Sdf, op->Htdf, sign, op->xsplit, op->Wh, op->Wl, (double2*)y,
                    (const double2*)bsub, pnrm);
}

// Start of a step (precision >= 1): precision 1 forms b = A_- psi and ||b||^2; precision 2 gets
// both the residual and ||b||^2 from the fused residual kernel, so nothing happens here.
void rhs_accurate(dirac_op* op, const void* psi)
{
    if (op->opts.precision == 2) {
        if (op->part_rdf) {
            k_set_int<<<1, 1, 0, op->st>>>(op->need_b, 1);
            op->launches++;
        }
        return;
    }
    Krylov& K = op->k64;
    apply_accurate(op, -1, psi, K.b, nullptr, op->part_n);
    finish(op, K.ks, 0, op->nparts_apply, nullptr, op->part_n, op->opts.max_iter);
}

// the owner pass's accumulators: fixed-binade form (offsets) or Dot2 (dirac_op_set_residual_mode)
static bool residual_offsets(const dirac_op* op)
{
    if (!op->own_sig) return false;
    return op->resid_mode == 2 || (op->resid_mode == 0 && op->opts.tol >= 1e-11);
}

// Refinement residual r = b - A_+ x, accurate to double precision, into k64.r, with the
// convergence check on k64.ks.  Precision 2: r = S (psi - x) - i tau H0 (psi + x) + (W - W^T)(psi + x)
// in one double-float pass, which also refreshes ||b||^2 = ||A_- psi||^2 (FP32 products).
void residual_accurate(dirac_op* op, const void* psi)
{
    Krylov& K = op->k64;
    if (op->opts.precision != 2) {
        apply_accurate(op, +1, K.x, K.r, K.b, op->part_n);
        finish(op, K.ks, 1, op->nparts_apply, nullptr, op->part_n, op->opts.max_iter);
        return;
    }
    if (op->part_rdf) {
        // owner/gather form: each coupling block read once
        {
            const bool off = residual_offsets(op);
            PhaseScope ps(op, DIRAC_PHASE_APPLY, off ? 6 : 4);   // split, [u sums, offsets,] owner (two), gather
            k_split_uv3<<<op->nparts_vec, 256, 0, op->st>>>(op->n, op->ov.n1, (const double2*)psi, (const double2*)K.x,
                                                           op->xsplit, op->vsplit, op->psi32);
            if (off)
                launch_residual_offsets(op->st, op->ov, op->asm_chunks, op->asm_nchunks, op->asm_gpair,
                                        op->asm_gcoef, op->s, op->own_E, op->own_Ew, op->own_US, op->own_sig,
                                        op->xsplit);
            {
                PhaseScope po(op, DIRAC_PHASE_OWNER, 0);   // the owner pass alone, inside the apply phase
                launch_residual_owner_df(op->st, op->ov, off, op->own_sig, op->xsplit, op->psi32, op->Wh, op->Wl,
                                         (double2*)K.r, op->b32, op->part_rdf, op->part_bdf, op->need_b,
                                         op->dev_err);
            }
            launch_residual_gather_df(op->st, op->ov, op->SdfT, op->HdfT, op->xsplit, op->vsplit, op->psi32,
                                      (double2*)K.r, op->b32, op->part_rdf, op->part_bdf, op->need_b, op->part_n,
                                      op->part_n2);
        }
        {
            PhaseScope ps(op, DIRAC_PHASE_VECTOR, 1);
            k_bnorm_if<<<1, 1024, 0, op->st>>>(K.ks, op->need_b, op->nparts_own, op->part_n2);
        }
        finish(op, K.ks, 1, op->nparts_own, nullptr, op->part_n, op->opts.max_iter);
        return;
    }
    {
        PhaseScope ps(op, DIRAC_PHASE_APPLY, 2);
        k_split_uv<<<op->nparts_vec, 256, 0, op->st>>>(op->n, (const double2*)psi, (const double2*)K.x, op->xsplit,
                                                      op->vsplit);
        launch_residual_df(dim3(op->ov.nch, grid_for(op->ov.n1, 128)), op->st, op->ov, op->Sdf, op->Htdf, op->xsplit,
                           op->vsplit, op->Wh, op->Wl, (double2*)K.r, op->part_n, op->part_n2);
    }
    finish(op, K.ks, 0, op->nparts_apply, nullptr, op->part_n2, op->opts.max_iter);
    finish(op, K.ks, 1, op->nparts_apply, nullptr, op->part_n, op->opts.max_iter);
}

void k_precond_launch(dirac_op* op, const Krylov& K, int mode, const KState* ks, const void* r,
                             const void* v, void* io, void* z, double* pn)
{
    PhaseScope ps(op, DIRAC_PHASE_PRECOND, 1);
    // schedule picked at setup: one lane per channel (channels of one kappa share the factor rows),
    // one warp per channel, or one warp per channel with the vector and the factor rows staged
    // through shared memory
    if (K.prec == 1) {
        if (op->prec_sched32 == 0 && op->prec_warps)
            launch_precond_lanes_t<float>(op->prec_warps, op->st, op->ov, K.Urow, K.L, K.Dinv, op->wks, op->wfirst,
                                          op->wcnt, mode, ks, r, v, io, z, pn);
        else if (op->prec_sched32 == 2 && op->prec_sm_ok)
            launch_precond_sm_t<float>(op->st, op->ov, K.U, K.L, K.Dinv, mode, ks, r, v, io, z, pn);
        else if (op->prec_sched32 == 3 && op->prec_rot_ok)
            launch_precond_rot_t<float>(op->st, op->ov, K.U, K.L, K.Dinv, mode, ks, r, v, io, z, pn);
        else
            launch_precond_t<float>(grid_for(op->ov.nch, 4), op->st, op->ov, K.U, K.L, K.Dinv, mode, ks, r, v, io, z,
                                    pn);
    } else {
        if (op->prec_sched64 == 2 && op->prec_sm_ok)
            launch_precond_sm_t<double>(op->st, op->ov, K.U, K.L, K.Dinv, mode, ks, r, v, io, z, pn);
        else if (op->prec_sched64 == 3 && op->prec_rot_ok)
            launch_precond_rot_t<double>(op->st, op->ov, K.U, K.L, K.Dinv, mode, ks, r, v, io, z, pn);
        else
            launch_precond_t<double>(grid_for(op->ov.nch, 4), op->st, op->ov, K.U, K.L, K.Dinv, mode, ks, r, v, io, z,
                                     pn);
    }
}

int prec_parts(const dirac_op* op, const Krylov& K)
{
    if (K.prec == 1) {
        if (op->prec_sched32 == 0 && op->prec_warps) return op->prec_warps;
        if (op->prec_sched32 == 2 && op->prec_sm_ok) return precond_sm_blocks<float>(op->ov.nch);
        if (op->prec_sched32 == 3 && op->prec_rot_ok) return precond_rot_blocks<float>(op->ov.nch);
        return grid_for(op->ov.nch, 4);
    }
    if (op->prec_sched64 == 2 && op->prec_sm_ok) return precond_sm_blocks<double>(op->ov.nch);
    if (op->prec_sched64 == 3 && op->prec_rot_ok) return precond_rot_blocks<double>(op->ov.nch);
    return grid_for(op->ov.nch, 4);
}

void finish(dirac_op* op, KState* ks, int what, int np, const double2* pd, const double* pn, int max_iter)
{
    PhaseScope ps(op, DIRAC_PHASE_VECTOR, 1);
    k_finish64<<<1, 1024, 0, op->st>>>(what, ks, np, pd, pn, nullptr, nullptr, max_iter);
}

void vcopy(dirac_op* op, const Krylov& K, const void* a, void* b)
{
    PhaseScope ps(op, DIRAC_PHASE_VECTOR, 1);
    if (K.prec == 0) k_copy64<<<op->nparts_vec, 256, 0, op->st>>>(op->n, (const double2*)a, (double2*)b);
    else k_copy32<<<op->nparts_vec, 256, 0, op->st>>>(op->n, (const float2*)a, (float2*)b);
}

void vzero(dirac_op* op, const Krylov& K, void* a)
{
    PhaseScope ps(op, DIRAC_PHASE_VECTOR, 1);
    if (K.prec == 0) k_zero64<<<op->nparts_vec, 256, 0, op->st>>>(op->n, (double2*)a);
    else k_zero32<<<op->nparts_vec, 256, 0, op->st>>>(op->n, (float2*)a);
}

dirac_status check_launch(const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return DIRAC_E_CUDA;
    }
    return DIRAC_OK;
}

// One BiCGSTAB iteration on K (right preconditioned); every launch is conditional on K.ks.  With
// mid_check the device state is read after the s-check, so a solve that converged there launches
// nothing more than the final update (large systems, where a host round trip is negligible).
dirac_status bicgstab_iteration(dirac_op* op, const Krylov& K, int max_iter, bool mid_check)
{
    int npa = apply_parts(op, K), npp = prec_parts(op, K), npv = op->nparts_vec;
    // p = r + beta (p - omega v); ph = M^-1 p
    k_precond_launch(op, K, 1, K.ks, K.r, K.v, K.p, K.ph, nullptr);
    // v = A ph, <rh, v>
    k_apply_launch(op, K, +1, K.ph, K.v, nullptr, K.rh, op->part_d, nullptr, K.ks);
    finish(op, K.ks, 2, npa, op->part_d, nullptr, max_iter);
    // s = r - alpha v; sh = M^-1 s; ||s||^2
    k_precond_launch(op, K, 2, K.ks, K.r, K.v, K.sv, K.sh, op->part_n);
    finish(op, K.ks, 3, npp, nullptr, op->part_n, max_iter);
    bool skip_t = false;
    if (mid_check) {
        KState hs;
        dirac_status e = read_state(op, K, hs);
        if (e) return e;
        skip_t = hs.done != 0;
    }
    if (!skip_t) {
        // t = A sh; <s, t>, ||t||^2 -> omega
        k_apply_launch(op, K, +1, K.sh, K.t, nullptr, K.sv, op->part_d, op->part_n, K.ks);
        finish(op, K.ks, 6, npa, op->part_d, op->part_n, max_iter);
    }
    // x += alpha ph + omega sh; r = s - omega t; <rh, r>, ||r||^2
    {
        PhaseScope ps(op, DIRAC_PHASE_VECTOR, 1);
        if (K.prec == 0)
            launch_update_xr_t<double>(npv, op->st, op->n, K.ks, K.x, K.r, K.ph, K.sh, K.sv, K.t, K.rh, op->part_d,
                                       op->part_n);
        else
            launch_update_xr_t<float>(npv, op->st, op->n, K.ks, K.x, K.r, K.ph, K.sh, K.sv, K.t, K.rh, op->part_d,
                                      op->part_n);
    }
    finish(op, K.ks, 5, npv, op->part_d, op->part_n, max_iter);
    return DIRAC_OK;
}

// r = b - A x (true residual) and a fresh Krylov start: rh = r, p = v = 0.  rel_start: the
// tolerance is relative to this starting residual (inner solves, zero initial guess).
void bicgstab_begin(dirac_op* op, const Krylov& K, int max_iter, bool rel_start)
{
    k_apply_launch(op, K, +1, K.x, K.r, K.b, nullptr, nullptr, op->part_n, nullptr);
    finish(op, K.ks, rel_start ? 8 : 1, apply_parts(op, K), nullptr, op->part_n, max_iter);
    vcopy(op, K, K.r, K.rh);
    vzero(op, K, K.p);
    vzero(op, K, K.v);
}

extern "C" dirac_status dirac_selftest_wait(dirac_op* op, double limit_cycles, int* timed_out)
{
    if (!op || !timed_out || !(limit_cycles >= 0) || limit_cycles > 4e9) {
        set_error("dirac_selftest_wait: bad argument");
        return DIRAC_E_ARG;
    }
    CUDA_TRY(cudaMemsetAsync(op->dev_err, 0, sizeof(int), op->st));
    CUDA_TRY(launch_wait_selftest(op->st, (long long)limit_cycles, op->dev_err));
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, op->dev_err, sizeof(int), cudaMemcpyDeviceToHost, op->st));
    CUDA_TRY(cudaStreamSynchronize(op->st));
    CUDA_TRY(cudaMemsetAsync(op->dev_err, 0, sizeof(int), op->st));
    *timed_out = h;
    return DIRAC_OK;
}

extern "C" dirac_status dirac_bounds_word(dirac_op* op, unsigned int* word, int* checked)
{
    if (!op || !word || !checked) {
        set_error("dirac_bounds_word: bad argument");
        return DIRAC_E_ARG;
    }
#ifdef DG_BOUNDS
    *checked = 1;
#else
    *checked = 0;
#endif
    unsigned int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, op->bounds_err, sizeof(h), cudaMemcpyDeviceToHost, op->st));
    CUDA_TRY(cudaStreamSynchronize(op->st));
    CUDA_TRY(cudaMemsetAsync(op->bounds_err, 0, sizeof(h), op->st));
    *word = h;
    return DIRAC_OK;
}

// the error word of kernels with bounded waits (synchronises the stream); cleared after reading
dirac_status check_dev_err(dirac_op* op, const char* what)
{
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, op->dev_err, sizeof(int), cudaMemcpyDeviceToHost, op->st));
    CUDA_TRY(cudaStreamSynchronize(op->st));
    if (!h) return DIRAC_OK;
    CUDA_TRY(cudaMemsetAsync(op->dev_err, 0, sizeof(int), op->st));
    set_error(std::string(what) + ": a kernel's bulk-copy wait ran out of time (results invalid)");
    return DIRAC_E_CUDA;
}

dirac_status read_state(dirac_op* op, const Krylov& K, KState& hs)
{
    CUDA_TRY(cudaMemcpyAsync(&hs, K.ks, sizeof(hs), cudaMemcpyDeviceToHost, op->st));
    CUDA_TRY(cudaStreamSynchronize(op->st));
    collect_phases(op);
    return DIRAC_OK;
}

// Iterate on K until the recursive residual meets K's tolerance (or a failure).  The device state
// is read after every `chunk` iterations; launches after convergence exit at once.
static dirac_status iterate(dirac_op* op, const Krylov& K, int max_iter, KState& hs)
{
    bool large = op->n > (1 << 20);   // large systems: host round trips cost nothing
    int chunk = large ? 1 : 4;
    for (;;) {
        for (int c = 0; c < chunk; c++) {
            dirac_status e = bicgstab_iteration(op, K, max_iter, large);
            if (e) return e;
        }
        dirac_status e = read_state(op, K, hs);
        if (e) return e;
        if (hs.done) return DIRAC_OK;
    }
}

// Solve A_+ x = b in K's precision to the tolerance in K.ks.  With true_check the solve ends only
// on the true residual (restarting on recursive-residual drift or breakdown); without it, on the
// recursive one.  Total iterations in *its.
static dirac_status solve(dirac_op* op, const Krylov& K, int max_iter, KState& hs, int* its, bool true_check)
{
    int total = 0, restarts = 0;
    for (;;) {
        bicgstab_begin(op, K, max_iter, !true_check && restarts == 0);
        dirac_status e = read_state(op, K, hs);
        if (e) return e;
        if (hs.status || hs.done) break;   // converged on the true residual (or failed)
        e = iterate(op, K, std::max(1, max_iter - total), hs);
        if (e) return e;
        total += hs.it;
        if (hs.status == 5 && restarts < 2) { restarts++; continue; }   // breakdown: restart from x
        if (hs.status) break;
        if (!true_check) break;
        if (total >= max_iter) { hs.status = 4; break; }
        if (++restarts > 8) { hs.status = 4; break; }
    }
    *its = total;
    return DIRAC_OK;
}

}  // namespace dg

using namespace dg;

extern "C" const char* dirac_last_error(void) { return g_err.c_str(); }

extern "C" void dirac_op_free(dirac_op* op)
{
    if (!op) return;
    cudaStreamSynchronize(op->st);
    if (op->st_asm) cudaStreamSynchronize(op->st_asm);
    collect_phases(op);
    graph_free(op);
    for (cudaEvent_t e : op->event_pool) cudaEventDestroy(e);
    for (auto& pe : op->pending) {
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    spec_free(op);
    if (op->ev_res) cudaEventDestroy(op->ev_res);
    for (int i = 0; i < 2; i++) {
        if (op->ev_asm[i]) cudaEventDestroy(op->ev_asm[i]);
        if (op->ev_use[i]) cudaEventDestroy(op->ev_use[i]);
    }
    if (op->st_asm) cudaStreamDestroy(op->st_asm);
    for (void* p : op->allocs) cudaFree(p);
    delete op;
}

extern "C" dirac_status dirac_profile(dirac_op* op, int enable)
{
    if (!op) { set_error("dirac_profile: NULL op"); return DIRAC_E_ARG; }
    CUDA_TRY(cudaStreamSynchronize(op->st));
    collect_phases(op);
    op->profiling = enable != 0;
    for (int i = 0; i < DIRAC_NPHASE; i++) { op->phase_ms[i] = 0; op->phase_n[i] = 0; }
    op->launches = 0;
    return DIRAC_OK;
}

extern "C" dirac_status dirac_profile_read(dirac_op* op, double* ms, int64_t* count, int64_t* launches)
{
    if (!op) { set_error("dirac_profile_read: NULL op"); return DIRAC_E_ARG; }
    CUDA_TRY(cudaStreamSynchronize(op->st));
    collect_phases(op);
    for (int i = 0; i < DIRAC_NPHASE; i++) {
        if (ms) ms[i] = op->phase_ms[i];
        if (count) count[i] = op->phase_n[i];
    }
    if (launches) *launches = op->launches;
    return DIRAC_OK;
}

extern "C" int64_t dirac_op_device_bytes(const dirac_op* op) { return op ? (int64_t)op->bytes : -1; }

// Preconditioner schedules, picked by timing: one lane per channel (the channels of one kappa share
// the factor rows read through shared memory), one warp per channel (more parallelism along the
// band), one warp per channel with the vector and factor rows staged through shared memory, or one
// warp per channel with each row fixed to a lane (one shuffle round per row, factor chunks only in
// shared memory).
// Which is fastest depends on the channel count and radial size, so the operator times one
// application of each on zeroed vectors (after a warm-up) and keeps the fastest, for the complex64
// inner solve and for the complex128 solve.  The choice does not change results beyond the solver
// tolerance (lane and warp substitutions round differently; the three warp kernels are identical).
static dirac_status time_precond(dirac_op* op, Krylov& K, int sched, float* ms)
{
    int& slot = K.prec == 1 ? op->prec_sched32 : op->prec_sched64;
    slot = sched;
    cudaEvent_t e[2];
    for (auto& ev : e) CUDA_TRY(cudaEventCreate(&ev));
    k_precond_launch(op, K, 0, nullptr, K.r, nullptr, nullptr, K.sh, nullptr);   // warm-up
    CUDA_TRY(cudaEventRecord(e[0], op->st));
    k_precond_launch(op, K, 0, nullptr, K.r, nullptr, nullptr, K.sh, nullptr);
    CUDA_TRY(cudaEventRecord(e[1], op->st));
    CUDA_TRY(cudaEventSynchronize(e[1]));
    CUDA_TRY(cudaEventElapsedTime(ms, e[0], e[1]));
    for (auto& ev : e) cudaEventDestroy(ev);
    return DIRAC_OK;
}

// Schedules chosen so far, per shape (radial slots, channels, precision of the solve, staged kernel
// available): operators of the same shape in one process take the same schedule, so their results
// agree bit for bit.
static std::mutex g_sched_mutex;
static std::map<std::tuple<int, int, int, int>, int> g_sched_cache;

static dirac_status tune_precond(dirac_op* op, Krylov& K)
{
    auto key = std::make_tuple(op->ov.n1, op->ov.nch, K.prec, (int)op->prec_sm_ok * 2 + (int)op->prec_rot_ok);
    {
        std::lock_guard<std::mutex> lock(g_sched_mutex);
        auto it = g_sched_cache.find(key);
        if (it != g_sched_cache.end()) {
            (K.prec == 1 ? op->prec_sched32 : op->prec_sched64) = it->second;
            return DIRAC_OK;
        }
    }
    size_t es = K.prec == 1 ? sizeof(float2) : sizeof(double2);
    CUDA_TRY(cudaMemsetAsync(K.r, 0, es * (size_t)op->n, op->st));
    CUDA_TRY(cudaMemsetAsync(K.sh, 0, es * (size_t)op->n, op->st));
    float* ms = K.prec == 1 ? op->prec_ms32 : op->prec_ms64;
    int best = -1;
    for (int sched = 0; sched < 4; sched++) {
        ms[sched] = 0;
        if (sched == 0 && (K.prec != 1 || !op->prec_warps)) continue;
        if (sched == 2 && !op->prec_sm_ok) continue;
        if (sched == 3 && !op->prec_rot_ok) continue;
        dirac_status e = time_precond(op, K, sched, &ms[sched]);
        if (e) return e;
        if (best < 0 || ms[sched] < ms[best]) best = sched;
    }
    (K.prec == 1 ? op->prec_sched32 : op->prec_sched64) = best;
    {
        std::lock_guard<std::mutex> lock(g_sched_mutex);
        g_sched_cache.emplace(key, best);
    }
    return check_launch("dirac_operator_setup: preconditioner schedule");
}

static dirac_status alloc_krylov(dirac_op* op, Krylov& K, int prec, double tol)
{
    size_t es = prec == 0 ? sizeof(double2) : sizeof(float2);
    void** vecs[] = {&K.b, &K.x, &K.r, &K.rh, &K.p, &K.v, &K.ph, &K.sv, &K.sh, &K.t};
    for (auto v : vecs) {
        char* p = nullptr;
        dirac_status s = dev_alloc(op, &p, (size_t)op->n * es);
        if (s) return s;
        *v = p;
    }
    dirac_status s = dev_alloc(op, &K.ks, 1);
    if (s) return s;
    KState k0{};
    k0.tol2 = tol * tol;
    CUDA_TRY(cudaMemcpy(K.ks, &k0, sizeof(k0), cudaMemcpyHostToDevice));
    K.prec = prec;
    return DIRAC_OK;
}

extern "C" dirac_status dirac_operator_setup(const dirac_basis* basis, const dirac_pulse* pulse,
                                             const dirac_solver_opts* opts, void* stream, dirac_op** out)
{
    if (!basis || !pulse || !opts || !out) { set_error("dirac_operator_setup: NULL argument"); return DIRAC_E_ARG; }
    if (!(opts->dt != 0) || !(opts->tol > 0) || opts->max_iter < 1 || !(pulse->omega > 0) ||
        !(pulse->n_cycles > 0) || opts->precision < 0 || opts->precision > 2 ||
        (opts->precision >= 1 && (!(opts->tol_inner > 0) || opts->tol_inner >= 1 || opts->max_outer < 1))) {
        set_error("dirac_operator_setup: invalid pulse or solver options");
        return DIRAC_E_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        set_error("dirac_operator_setup: no CUDA device");
        return DIRAC_E_STATE;
    }
    dirac_op* op = new dirac_op();
    op->B = basis->b;
    op->pulse = *pulse;
    op->opts = *opts;
    op->st = (cudaStream_t)stream;
    cudaGetDevice(&op->device);
    const Basis& B = op->B;
    int n1 = B.n1, bd = B.bd, half = B.half, nk2 = 2 * B.p.kappa_max;
    bool mixed = opts->precision >= 1;
    bool dfloat = opts->precision == 2;
    op->n = B.n();
    op->npairs = (int64_t)B.pa.size();
    double tau = 0.5 * opts->dt;
    dirac_status s = DIRAC_OK;
#define TRY(x)                                  \
    do {                                        \
        s = (x);                                \
        if (s) { dirac_op_free(op); return s; } \
    } while (0)

    // radial blocks per kappa
    std::vector<double> hS((size_t)nk2 * n1 * bd * 4), hH(hS.size());
    for (int ks = 0; ks < nk2; ks++) {
        int kappa = (ks % 2 ? 1 : -1) * (ks / 2 + 1);
        Band Sb, Hb;
        radial_blocks(B, kappa, Sb, Hb);
        std::copy(Sb.v.begin(), Sb.v.end(), hS.begin() + (size_t)ks * n1 * bd * 4);
        std::copy(Hb.v.begin(), Hb.v.end(), hH.begin() + (size_t)ks * n1 * bd * 4);
    }
    double *dS, *dH;
    TRY(upload(op, &dS, hS));
    TRY(upload(op, &dH, hH));
    std::vector<int> kslot(B.nch);
    for (int a = 0; a < B.nch; a++) kslot[a] = kappa_slot(B.kap[a]);
    int *dks, *dkap;
    TRY(upload(op, &dks, kslot));
    TRY(upload(op, &dkap, B.kap));
    TRY(upload(op, &op->ch_two_mu, B.tmu));

    // adjacency: per channel, pairs where it is the lower channel (W x) or the upper one (W^T x)
    std::vector<std::vector<int>> adjp(B.nch), adjn(B.nch), adjt(B.nch);
    for (int64_t q = 0; q < op->npairs; q++) {
        int a = B.pa[q], b = B.pb[q];
        adjp[a].push_back((int)q); adjn[a].push_back(b); adjt[a].push_back(0);
        adjp[b].push_back((int)q); adjn[b].push_back(a); adjt[b].push_back(1);
    }
    std::vector<int> as(1, 0), ap, an, at;
    for (int a = 0; a < B.nch; a++) {
        ap.insert(ap.end(), adjp[a].begin(), adjp[a].end());
        an.insert(an.end(), adjn[a].begin(), adjn[a].end());
        at.insert(at.end(), adjt[a].begin(), adjt[a].end());
        as.push_back((int)ap.size());
    }
    // owner lists (pairs a channel is the lower channel of) and in-lists (upper channel of), for the
    // apply that reads each coupling block once
    std::vector<int> ows(1, 0), owp, own, ins(1, 0), inp;
    for (int a = 0; a < B.nch; a++) {
        for (size_t k = 0; k < adjp[a].size(); k++) {
            if (adjt[a][k] == 0) { owp.push_back(adjp[a][k]); own.push_back(adjn[a][k]); }
            else inp.push_back(adjp[a][k]);
        }
        ows.push_back((int)owp.size());
        ins.push_back((int)inp.size());
    }
    int *dows, *dowp, *down, *dins, *dinp;
    TRY(upload(op, &dows, ows));
    TRY(upload(op, &dowp, owp));
    TRY(upload(op, &down, own));
    TRY(upload(op, &dins, ins));
    TRY(upload(op, &dinp, inp));
    int *das, *dap, *dan, *dat, *dpa, *dpb, *dts, *dtl;
    TRY(upload(op, &das, as));
    TRY(upload(op, &dap, ap));
    TRY(upload(op, &dan, an));
    TRY(upload(op, &dat, at));
    TRY(upload(op, &dpa, B.pa));
    TRY(upload(op, &dpb, B.pb));
    TRY(upload(op, &dts, B.pterm_start));
    // pair terms: cA[n] = -c tau A1 m_n(ka, kb), cB[n] = c tau A2 m_n(kb, ka), m = (1, k', k, k'k)
    std::vector<int> tl(B.pterm.size());
    std::vector<double> tc(B.pterm.size() * 8);
    for (int64_t q = 0; q < op->npairs; q++) {
        double ka = B.kap[B.pa[q]], kb = B.kap[B.pb[q]];
        double mab[4] = {1, ka, kb, ka * kb}, mba[4] = {1, kb, ka, ka * kb};
        for (int e = B.pterm_start[q]; e < B.pterm_start[q + 1]; e++) {
            tl[e] = B.pterm[e].l;
            for (int nn = 0; nn < 4; nn++) {
                tc[(size_t)e * 8 + nn] = -B.p.c * tau * B.pterm[e].A1 * mab[nn];
                tc[(size_t)e * 8 + 4 + nn] = B.p.c * tau * B.pterm[e].A2 * mba[nn];
            }
        }
    }
    double* dtc;
    TRY(upload(op, &dtl, tl));
    TRY(upload(op, &dtc, tc));
    // distinct (k', k, l) bands and per-term references to them
    std::vector<int> keyl, tkd(B.pterm.size()), tkt(B.pterm.size());
    std::vector<double> keym, tcab(2 * B.pterm.size());
    std::vector<int> index((size_t)nk2 * nk2 * (B.p.l_max + 1), -1);
    auto key_index = [&](int kp, int k, int l) {
        return index[((size_t)kappa_slot(kp) * nk2 + kappa_slot(k)) * (B.p.l_max + 1) + l];
    };
    {
        auto key_of = [&](int kp, int k, int l) {
            size_t id = ((size_t)kappa_slot(kp) * nk2 + kappa_slot(k)) * (B.p.l_max + 1) + l;
            if (index[id] < 0) {
                index[id] = (int)keyl.size();
                keyl.push_back(l);
                keym.insert(keym.end(), {1.0, (double)kp, (double)k, (double)kp * k});
            }
            return index[id];
        };
        for (int64_t q = 0; q < op->npairs; q++) {
            int ka = B.kap[B.pa[q]], kb = B.kap[B.pb[q]];
            for (int e = B.pterm_start[q]; e < B.pterm_start[q + 1]; e++) {
                tkd[e] = key_of(ka, kb, B.pterm[e].l);
                tkt[e] = key_of(kb, ka, B.pterm[e].l);
                tcab[2 * e] = -B.p.c * tau * B.pterm[e].A1;
                tcab[2 * e + 1] = B.p.c * tau * B.pterm[e].A2;
            }
        }
    }
    std::vector<int> porder(op->npairs);
    for (int64_t q = 0; q < op->npairs; q++) porder[q] = (int)q;
    std::stable_sort(porder.begin(), porder.end(), [&](int x, int y) {
        int kx = kappa_slot(B.kap[B.pa[x]]) * nk2 + kappa_slot(B.kap[B.pb[x]]);
        int ky = kappa_slot(B.kap[B.pa[y]]) * nk2 + kappa_slot(B.kap[B.pb[y]]);
        return kx < ky;
    });
    int *dkl, *dkd, *dkt, *dpo;
    double *dkm, *dcab;
    TRY(upload(op, &dkl, keyl));
    TRY(upload(op, &dkm, keym));
    TRY(upload(op, &dkd, tkd));
    TRY(upload(op, &dkt, tkt));
    TRY(upload(op, &dcab, tcab));
    TRY(upload(op, &dpo, porder));

    // preconditioner factors, one per radial block
    int kb = 2 * half + 1, ns = 2 * n1, wu = 2 * kb;
    std::vector<double2> hU((size_t)nk2 * ns * (wu + 1)), hL((size_t)nk2 * ns * kb);
    std::vector<double2> hUr((size_t)nk2 * ns * (wu + 1)), hDi((size_t)nk2 * ns);
    std::vector<int> hP((size_t)nk2 * ns);
    for (int ks = 0; ks < nk2; ks++) {
        int kappa = (ks % 2 ? 1 : -1) * (ks / 2 + 1);
        BandLU<cd> lu;
        if (!precond_factor(B, kappa, tau, lu)) {
            set_error("dirac_operator_setup: singular preconditioner block");
            dirac_op_free(op);
            return DIRAC_E_NUMERIC;
        }
        // column form for the back substitution: Ucol[i][k] = U[i-k][k] (zero above the first row)
        for (int i = 0; i < ns; i++)
            for (int k = 0; k <= wu; k++) {
                cd u = i - k >= 0 ? lu.U[(size_t)(i - k) * (wu + 1) + k] : cd(0);
                hU[((size_t)ks * ns + i) * (wu + 1) + k] = make_double2(u.real(), u.imag());
            }
        for (size_t e = 0; e < lu.U.size(); e++)
            hUr[(size_t)ks * ns * (wu + 1) + e] = make_double2(lu.U[e].real(), lu.U[e].imag());
        for (int i = 0; i < ns; i++) {
            cd di = cd(1.0) / lu.U[(size_t)i * (wu + 1)];
            hDi[(size_t)ks * ns + i] = make_double2(di.real(), di.imag());
        }
        for (size_t e = 0; e < lu.L.size(); e++)
            hL[(size_t)ks * ns * kb + e] = make_double2(lu.L[e].real(), lu.L[e].imag());
        std::copy(lu.piv.begin(), lu.piv.end(), hP.begin() + (size_t)ks * ns);
    }
    double2 *dU, *dL, *dUr, *dDi;
    int *dP, *dord;
    TRY(upload(op, &dU, hU));
    TRY(upload(op, &dL, hL));
    TRY(upload(op, &dUr, hUr));
    TRY(upload(op, &dDi, hDi));
    TRY(upload(op, &dP, hP));
    std::vector<int> ord(B.nch);
    for (int a = 0; a < B.nch; a++) ord[a] = a;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return kslot[x] < kslot[y]; });
    TRY(upload(op, &dord, ord));
    // same-kappa groups of at most 32 channels for the lane-per-channel preconditioner
    if (kb == 13) {
        std::vector<int> wk, wf, wc;
        for (int i = 0; i < B.nch;) {
            int j = i;
            while (j < B.nch && kslot[ord[j]] == kslot[ord[i]] && j - i < 32) j++;
            wk.push_back(kslot[ord[i]]);
            wf.push_back(i);
            wc.push_back(j - i);
            i = j;
        }
        op->prec_warps = (int)wk.size();
        TRY(upload(op, &op->wks, wk));
        TRY(upload(op, &op->wfirst, wf));
        TRY(upload(op, &op->wcnt, wc));
    }

    // pulse matrices
    PulseData P;
    pulse_matrices(B, *pulse, P);
    size_t be = (size_t)n1 * bd * 4;
    std::vector<double> hM((size_t)P.L * 3 * 4 * be);
    for (size_t gi = 0; gi < P.g.size(); gi++) std::copy(P.g[gi].v.begin(), P.g[gi].v.end(), hM.begin() + gi * be);
    double* dM;
    TRY(upload(op, &dM, hM));
    TRY(dev_alloc(op, &op->G, (size_t)P.L * 4 * be));
    TRY(dev_alloc(op, &op->s, (size_t)P.L * 3));
    TRY(dev_alloc(op, &op->t_eval, 1));
    if (!dfloat) {
        TRY(dev_alloc(op, &op->W, (size_t)std::max<int64_t>(op->npairs, 1) * be));
        TRY(dev_alloc(op, &op->K, (size_t)std::max<size_t>(keyl.size(), 1) * be));
    } else {
        auto split = [](double v) { float h = (float)v; return make_float2(h, (float)(v - (double)h)); };
        std::vector<float2> sdf(hS.size()), hdf(hH.size());
        for (size_t e = 0; e < hS.size(); e++) { sdf[e] = split(hS[e]); hdf[e] = split(tau * hH[e]); }
        TRY(upload(op, &op->Sdf, sdf));
        TRY(upload(op, &op->Htdf, hdf));
        if (bd == 13) {
            // the same bands with the rows innermost, [kappa slot][d][row][entry], for the residual's
            // gather pass (its threads hold consecutive rows: a diagonal's 2 x 2 block of a row is one
            // 32-byte record next to the neighbouring rows' records)
            std::vector<float2> st(sdf.size()), ht(hdf.size());
            for (int ks = 0; ks < nk2; ks++)
                for (int r = 0; r < n1; r++)
                    for (int d = 0; d < bd; d++)
                        for (int e = 0; e < 4; e++) {
                            size_t a = (((size_t)ks * n1 + r) * bd + d) * 4 + e;
                            size_t t = (((size_t)ks * bd + d) * n1 + r) * 4 + e;
                            st[t] = sdf[a];
                            ht[t] = hdf[a];
                        }
            TRY(upload(op, &op->SdfT, st));
            TRY(upload(op, &op->HdfT, ht));
        }
        std::vector<float4> cdf(B.pterm.size());
        for (size_t e = 0; e < cdf.size(); e++) {
            float2 a = split(tcab[2 * e]), b = split(tcab[2 * e + 1]);
            cdf[e] = make_float4(a.x, a.y, b.x, b.y);
        }
        TRY(upload(op, &op->cab_df, cdf));
        // pair groups (same kappa_a, kappa_b; adjacent in porder) in chunks of at most ASM_CHUNK pairs
        {
            std::vector<AsmChunk> chunks;
            std::vector<int> gpair;
            std::vector<float4> gcoef;
            bool ok = true;
            for (int64_t i = 0; i < op->npairs && ok;) {
                int q0 = porder[i];
                int ka = B.kap[B.pa[q0]], kb = B.kap[B.pb[q0]];
                int64_t j = i;
                while (j < op->npairs && B.kap[B.pa[porder[j]]] == ka && B.kap[B.pb[porder[j]]] == kb) j++;
                std::vector<int> ls;
                for (int64_t u = i; u < j; u++)
                    for (int e = B.pterm_start[porder[u]]; e < B.pterm_start[porder[u] + 1]; e++)
                        if (std::find(ls.begin(), ls.end(), B.pterm[e].l) == ls.end()) ls.push_back(B.pterm[e].l);
                std::sort(ls.begin(), ls.end());
                if ((int)ls.size() > ASM_MAX_NL) { ok = false; break; }
                int64_t cnt = j - i, nchk = (cnt + ASM_CHUNK - 1) / ASM_CHUNK;
                for (int64_t c = 0; c < nchk; c++) {
                    int64_t c0 = i + cnt * c / nchk, c1 = i + cnt * (c + 1) / nchk;
                    AsmChunk ch{};
                    ch.first = (int)gpair.size();
                    ch.count = (int)(c1 - c0);
                    ch.nl = (int)ls.size();
                    ch.ka = ka;
                    ch.kb = kb;
                    for (int m = 0; m < ASM_MAX_NL; m++) ch.l[m] = m < ch.nl ? ls[m] : ls[0];
                    chunks.push_back(ch);
                    for (int64_t u = c0; u < c1; u++) {
                        int q = porder[u];
                        gpair.push_back(q);
                        size_t base = gcoef.size();
                        gcoef.resize(base + ASM_MAX_NL, make_float4(0.f, 0.f, 0.f, 0.f));
                        for (int e = B.pterm_start[q]; e < B.pterm_start[q + 1]; e++) {
                            int m = (int)(std::find(ls.begin(), ls.end(), B.pterm[e].l) - ls.begin());
                            gcoef[base + m] = cdf[e];
                        }
                    }
                }
                i = j;
            }
            if (ok && !chunks.empty()) {
                op->asm_nchunks = (int)chunks.size();
                TRY(upload(op, &op->asm_chunks, chunks));
                TRY(upload(op, &op->asm_gpair, gpair));
                TRY(upload(op, &op->asm_gcoef, gcoef));
            }
        }
        TRY(dev_alloc(op, &op->Gdf, (size_t)P.L * 4 * be));
        if (!op->asm_chunks) {   // the per-pair assembly reads combined K bands; the grouped one forms them
            TRY(dev_alloc(op, &op->Kdf, (size_t)std::max<size_t>(keyl.size(), 1) * be));
            TRY(dev_alloc(op, &op->KTdf, (size_t)std::max<size_t>(keyl.size(), 1) * be));
        }
        TRY(dev_alloc(op, &op->Wh, (size_t)std::max<int64_t>(op->npairs, 1) * be));
        TRY(dev_alloc(op, &op->Wl, (size_t)std::max<int64_t>(op->npairs, 1) * be));
        TRY(dev_alloc(op, &op->xsplit, (size_t)op->n));
        TRY(dev_alloc(op, &op->vsplit, (size_t)op->n));
        op->aset[0] = AsmSet{op->t_eval, op->s, op->Gdf, op->Kdf, op->KTdf, op->Wh, op->Wl};
        op->acur = 0;
    }

    // Krylov workspaces and reduction partials
    TRY(alloc_krylov(op, op->k64, 0, opts->tol));
    op->k64.S = dS; op->k64.H = dH; op->k64.W = op->W; op->k64.U = dU; op->k64.L = dL;
    op->k64.Urow = dUr; op->k64.Dinv = dDi;
    if (mixed) {
        if (!dfloat) TRY(dev_alloc(op, &op->W32, (size_t)std::max<int64_t>(op->npairs, 1) * be));
        TRY(alloc_krylov(op, op->k32, 1, opts->tol_inner));
        std::vector<float> fS(hS.begin(), hS.end()), fH(hH.begin(), hH.end());
        auto tof = [](const std::vector<double2>& a) {
            std::vector<float2> f(a.size());
            for (size_t e = 0; e < a.size(); e++) f[e] = make_float2((float)a[e].x, (float)a[e].y);
            return f;
        };
        std::vector<float2> fU = tof(hU), fL = tof(hL), fUr = tof(hUr), fDi = tof(hDi);
        float *fdS, *fdH;
        float2 *fdU, *fdL, *fdUr, *fdDi;
        TRY(upload(op, &fdS, fS));
        TRY(upload(op, &fdH, fH));
        if (bd == 13) {
            // rows innermost, [kappa slot][d][row][entry], for the complex64 owner pass's diagonal block
            std::vector<float> st(fS.size()), ht(fH.size());
            for (int ks = 0; ks < nk2; ks++)
                for (int r = 0; r < n1; r++)
                    for (int d = 0; d < bd; d++)
                        for (int e = 0; e < 4; e++) {
                            size_t a = (((size_t)ks * n1 + r) * bd + d) * 4 + e;
                            size_t t = (((size_t)ks * bd + d) * n1 + r) * 4 + e;
                            st[t] = fS[a];
                            ht[t] = fH[a];
                        }
            TRY(upload(op, &op->S32T, st));
            TRY(upload(op, &op->H32T, ht));
        }
        TRY(upload(op, &fdU, fU));
        TRY(upload(op, &fdL, fL));
        TRY(upload(op, &fdUr, fUr));
        TRY(upload(op, &fdDi, fDi));
        op->k32.Urow = fdUr; op->k32.Dinv = fdDi;
        op->k32.S = fdS; op->k32.H = fdH; op->k32.W = dfloat ? (const void*)op->Wh : (const void*)op->W32;
        op->k32.U = fdU; op->k32.L = fdL;
        if (bd == 13 && op->npairs) {
            // partial transposed products of the owner/gather apply
            int ntile = grid_for(n1, apply_own_tile());
            size_t nslot = (size_t)op->npairs * ntile * apply_own_nout();
            TRY(dev_alloc(op, &op->part_own, nslot));
            if (dfloat) {
                TRY(dev_alloc(op, &op->part_rdf, 2 * nslot));
                TRY(dev_alloc(op, &op->part_bdf, nslot));
                // envelopes for the owner pass's accumulator offsets (grouped assembly only):
                // E[l][n][r] = the largest |M_lcn| entry (over c and the 2 x 2 block) of row r and of
                // column r (rows rr with rr + d - h = r); Ew = its maximum over rows r - h .. r + h.
                // Rounded up.
                if (op->asm_chunks) {
                    std::vector<float> hE((size_t)P.L * 4 * n1, 0.f), hEw(hE.size(), 0.f);
                    for (int l = 0; l < P.L; l++)
                        for (int nn = 0; nn < 4; nn++) {
                            std::vector<double> env(n1, 0.0);
                            for (int cc = 0; cc < 3; cc++) {
                                const double* g = hM.data() + ((size_t)(l * 3 + cc) * 4 + nn) * be;
                                for (int r = 0; r < n1; r++)
                                    for (int d = 0; d < bd; d++) {
                                        double m = 0;
                                        for (int e = 0; e < 4; e++)
                                            m = std::max(m, std::fabs(g[((size_t)r * bd + d) * 4 + e]));
                                        env[r] = std::max(env[r], m);
                                        int rr = r + d - half;
                                        if (rr >= 0 && rr < n1) env[rr] = std::max(env[rr], m);
                                    }
                            }
                            float* Er = hE.data() + ((size_t)l * 4 + nn) * n1;
                            float* Ewr = hEw.data() + ((size_t)l * 4 + nn) * n1;
                            for (int r = 0; r < n1; r++) Er[r] = (float)(env[r] * (1.0 + 1e-6));
                            for (int r = 0; r < n1; r++) {
                                float m = 0.f;
                                for (int rr = std::max(0, r - half); rr <= std::min(n1 - 1, r + half); rr++)
                                    m = std::max(m, Er[rr]);
                                Ewr[r] = m;
                            }
                        }
                    TRY(upload(op, &op->own_E, hE));
                    TRY(upload(op, &op->own_Ew, hEw));
                    // u-window sums with zero margins (residual_us_floats); the margins stay zero
                    const size_t nus = residual_us_floats(B.nch, n1);
                    TRY(dev_alloc(op, &op->own_US, nus));
                    if (cudaMemsetAsync(op->own_US, 0, nus * sizeof(float), op->st) != cudaSuccess) {
                        set_error("dirac_operator_setup: cudaMemsetAsync failed");
                        dirac_op_free(op);
                        return DIRAC_E_CUDA;
                    }
                    TRY(dev_alloc(op, &op->own_sig, (size_t)op->npairs * ntile * residual_sig_bytes()));
                }
                TRY(dev_alloc(op, &op->psi32, (size_t)op->n));
                TRY(dev_alloc(op, &op->b32, (size_t)op->n));
                TRY(dev_alloc(op, &op->need_b, 1));
                if (cudaMemsetAsync(op->need_b, 0, sizeof(int), op->st) != cudaSuccess) {
                    set_error("dirac_operator_setup: cudaMemsetAsync failed");
                    dirac_op_free(op);
                    return DIRAC_E_CUDA;
                }
            }
            cudaError_t ce = apply_own32_prepare();
            if (ce != cudaSuccess) {
                set_error(std::string("dirac_operator_setup: ") + cudaGetErrorString(ce));
                dirac_op_free(op);
                return DIRAC_E_CUDA;
            }
        }
    }
    op->nparts_apply = grid_for(n1, 128) * B.nch;
    op->nparts_own = grid_for(n1, apply_own_tile()) * B.nch;
    op->nparts_vec = grid_for(op->n, 256);
    op->nparts_prec = grid_for(B.nch, 4);                     // ||s||^2 partials, warp-per-channel kernel
    op->nparts_prec32 = op->prec_warps ? op->prec_warps : grid_for(B.nch, 4);   // lane-per-channel kernel
    int np = std::max({op->nparts_apply, op->nparts_own, op->nparts_vec, op->nparts_prec, op->nparts_prec32,
                       grid_for(n1, FTR) * B.nch,
                       precond_sm_blocks<double>(B.nch), precond_sm_blocks<float>(B.nch),
                       precond_rot_blocks<double>(B.nch), precond_rot_blocks<float>(B.nch)});
    TRY(dev_alloc(op, &op->part_d, (size_t)np));
    TRY(dev_alloc(op, &op->part_d2, (size_t)np));
    TRY(dev_alloc(op, &op->part_n, (size_t)np));
    TRY(dev_alloc(op, &op->part_n2, (size_t)np));
    TRY(dev_alloc(op, &op->dev_err, 1));
    TRY(dev_alloc(op, &op->bounds_err, 1));
    if (cudaMemsetAsync(op->dev_err, 0, sizeof(int), op->st) != cudaSuccess ||
        cudaMemsetAsync(op->bounds_err, 0, sizeof(unsigned int), op->st) != cudaSuccess) {
        set_error("dirac_operator_setup: cudaMemsetAsync failed");
        dirac_op_free(op);
        return DIRAC_E_CUDA;
    }
    // ground state of the kappa = -1, mu = +1/2 channel for the observables
    for (int a = 0; a < B.nch; a++)
        if (B.kap[a] == -1 && B.tmu[a] == 1) op->ground_ch = a;
    std::vector<double2> g0(2 * n1);
    if (op->ground_ch >= 0)
        for (int i = 0; i < 2 * n1; i++)
            g0[i] = make_double2(B.psi0[((size_t)op->ground_ch * 2 * n1 + i) * 2],
                                 B.psi0[((size_t)op->ground_ch * 2 * n1 + i) * 2 + 1]);
    TRY(upload(op, &op->psi0_g, g0));

    OpView& o = op->ov;
    o.n1 = n1; o.bd = bd; o.half = half; o.nch = B.nch; o.npairs = op->npairs; o.tau = tau; o.c = B.p.c;
    o.ch_kslot = dks; o.ch_kappa = dkap; o.S = dS; o.H = dH;
    o.adj_start = das; o.adj_pair = dap; o.adj_nbr = dan; o.adj_tr = dat;
    o.own_start = dows; o.own_pair = dowp; o.own_nbr = down; o.in_start = dins; o.in_pair = dinp;
    o.pair_a = dpa; o.pair_b = dpb; o.term_start = dts; o.term_l = dtl; o.term_coef = dtc;
    o.nkeys = (int)keyl.size(); o.key_l = dkl; o.key_mono = dkm; o.term_kd = dkd; o.term_kt = dkt;
    o.term_cab = dcab; o.pair_order = dpo;
    o.bounds_err = op->bounds_err;
    o.nb_part = op->part_own ? (int64_t)op->npairs * grid_for(n1, apply_own_tile()) * apply_own_nout() : 0;
    o.nb_coup = (int64_t)op->npairs * n1 * bd * 4;
    o.kb = kb; o.luU = dU; o.luL = dL; o.luP = dP; o.prec_order = dord;
    PulseView& pv = op->pv;
    pv.L = P.L; pv.T = P.T; pv.amp = P.amp; pv.t0 = pulse->t0; pv.dt = opts->dt;
    for (int c = 0; c < 3; c++) { pv.w[c] = P.w[c]; pv.wt[c] = P.wt[c]; }
    pv.M = dM;
    // the staged and rotated-lane kernels are built for 13 block-diagonals (order-7 splines)
    op->prec_sm_ok = bd == 13 && precond_sm_prepare<float>(n1) == cudaSuccess &&
                     precond_sm_prepare<double>(n1) == cudaSuccess;
    cudaGetLastError();
    op->prec_rot_ok = bd == 13 && precond_rot_prepare<float>() == cudaSuccess &&
                      precond_rot_prepare<double>() == cudaSuccess;
    cudaGetLastError();
    {
        dirac_status ts = tune_precond(op, op->k64);
        if (!ts && mixed) ts = tune_precond(op, op->k32);
        if (ts) { dirac_op_free(op); return ts; }
    }
    {
        // the device address of dirac_observables_static's scratch, looked up here so that call
        // does no set-up; a failure is reported by that call (it retries), not by the setup
        double2* scratch = nullptr;
        if (obs_scratch_address(op->device, &scratch) != DIRAC_OK) cudaGetLastError();
    }
    *out = op;
#undef TRY
    return DIRAC_OK;
}

extern "C" dirac_status dirac_apply(dirac_op* op, int sign, double t, const void* x_dev, void* y_dev)
{
    if (!op || !x_dev || !y_dev || x_dev == y_dev || (sign != 1 && sign != -1)) {
        set_error("dirac_apply: bad argument");
        return DIRAC_E_ARG;
    }
    k_set_time<<<1, 1, 0, op->st>>>(op->t_eval, t);
    op->launches++;
    launch_assemble(op);
    apply_accurate(op, sign, x_dev, y_dev, nullptr, nullptr);
    return check_launch("dirac_apply");
}

extern "C" dirac_status dirac_apply_assembled(dirac_op* op, int sign, const void* x_dev, void* y_dev)
{
    if (!op || !x_dev || !y_dev || x_dev == y_dev || (sign != 1 && sign != -1)) {
        set_error("dirac_apply_assembled: bad argument");
        return DIRAC_E_ARG;
    }
    apply_accurate(op, sign, x_dev, y_dev, nullptr, nullptr);
    return check_launch("dirac_apply_assembled");
}

extern "C" dirac_status dirac_precond_apply(dirac_op* op, const void* r_dev, void* z_dev)
{
    if (!op || !r_dev || !z_dev || r_dev == z_dev) { set_error("dirac_precond_apply: bad argument"); return DIRAC_E_ARG; }
    k_precond_launch(op, op->k64, 0, nullptr, r_dev, nullptr, nullptr, z_dev, nullptr);
    return check_launch("dirac_precond_apply");
}

extern "C" dirac_status dirac_apply32(dirac_op* op, int sign, double t, const void* x_dev, void* y_dev)
{
    if (!op || !x_dev || !y_dev || x_dev == y_dev || (sign != 1 && sign != -1)) {
        set_error("dirac_apply32: bad argument");
        return DIRAC_E_ARG;
    }
    if (op->opts.precision == 0 || !op->k32.ks) {
        set_error("dirac_apply32: the complex64 operator exists in precision 1 and 2 only");
        return DIRAC_E_ARG;
    }
    k_set_time<<<1, 1, 0, op->st>>>(op->t_eval, t);
    op->launches++;
    launch_assemble(op);
    k_apply_launch(op, op->k32, sign, x_dev, y_dev, nullptr, nullptr, nullptr, nullptr, nullptr);
    dirac_status e = check_launch("dirac_apply32");
    if (e) return e;
    return check_dev_err(op, "dirac_apply32");
}

extern "C" dirac_status dirac_precond_apply32(dirac_op* op, const void* r_dev, void* z_dev)
{
    if (!op || !r_dev || !z_dev || r_dev == z_dev) { set_error("dirac_precond_apply32: bad argument"); return DIRAC_E_ARG; }
    if (op->opts.precision == 0 || !op->k32.ks) {
        set_error("dirac_precond_apply32: the complex64 preconditioner exists in precision 1 and 2 only");
        return DIRAC_E_ARG;
    }
    k_precond_launch(op, op->k32, 0, nullptr, r_dev, nullptr, nullptr, z_dev, nullptr);
    return check_launch("dirac_precond_apply32");
}

extern "C" dirac_status dirac_residual(dirac_op* op, double t, const void* psi_dev, const void* x_dev, void* r_dev,
                                       double* bnorm)
{
    if (!op || !psi_dev || !x_dev || !r_dev || r_dev == psi_dev || r_dev == x_dev) {
        set_error("dirac_residual: bad argument");
        return DIRAC_E_ARG;
    }
    Krylov& K = op->k64;
    k_set_time<<<1, 1, 0, op->st>>>(op->t_eval, t);
    op->launches++;
    launch_assemble(op);
    vcopy(op, K, x_dev, K.x);
    // b = A_- psi and ||b||^2 (precision 2 forms both inside the residual pass), then r = b - A_+ x
    if (op->opts.precision == 0) {
        apply_accurate(op, -1, psi_dev, K.b, nullptr, op->part_n);
        finish(op, K.ks, 0, op->nparts_apply, nullptr, op->part_n, op->opts.max_iter);
    } else {
        rhs_accurate(op, psi_dev);
    }
    residual_accurate(op, psi_dev);
    vcopy(op, K, K.r, r_dev);
    dirac_status e = check_launch("dirac_residual");
    if (e) return e;
    KState hs;
    e = read_state(op, K, hs);
    if (e) return e;
    if (bnorm) *bnorm = std::sqrt(hs.bnorm2);
    return check_dev_err(op, "dirac_residual");
}

extern "C" dirac_status dirac_op_set_schedule(dirac_op* op, int complex64, int sched)
{
    if (!op || sched < 0 || sched > 3 || (sched == 0 && (!complex64 || !op->prec_warps)) ||
        (sched == 2 && !op->prec_sm_ok) || (sched == 3 && !op->prec_rot_ok) || (complex64 && !op->k32.ks)) {
        set_error("dirac_op_set_schedule: schedule not available for this operator");
        return DIRAC_E_ARG;
    }
    (complex64 ? op->prec_sched32 : op->prec_sched64) = sched;
    op->config_gen++;   // captured graphs hold the old kernel
    return DIRAC_OK;
}

// Subgroup form of the factorised apply (mode 1): kappa chunks of up to FLANE channels for the radial
// pass; for the angular pass, the channels of each mu in FSG-sized subgroups (ordered by the parity
// of their orbital l, then |kappa|, so that a subgroup's outputs share many partners) with the union
// of their (partner, multipole) items and per item and output the coefficients of U, V, U', V'
// (own pairs a < b: -(cA, cA ka, cB, cB ka); pairs b < a: (cB, cB ka, cA, cA ka); the apply's sign
// is applied in the kernel).
static dirac_status fact_sub_setup(dirac_op* op)
{
    using namespace dg;
    const Basis& B = op->B;
    const int nch = B.nch, L = op->pv.L;
    // radial: kappa groups of the kappa-sorted channel order, FLANE channels at a time
    std::vector<int> ks(nch), ordv(nch);
    CUDA_TRY(cudaMemcpy(ordv.data(), op->ov.prec_order, sizeof(int) * nch, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(ks.data(), op->ov.ch_kslot, sizeof(int) * nch, cudaMemcpyDeviceToHost));
    std::vector<RadChunk> ch1;
    for (int i = 0; i < nch;) {
        int j = i;
        while (j < nch && ks[ordv[j]] == ks[ordv[i]] && j - i < FLANE) j++;
        ch1.push_back(RadChunk{ks[ordv[i]], B.kap[ordv[i]], i, j - i});
        i = j;
    }
    // two chunks per block where their channels fit the lanes together: largest first, each paired
    // with the largest unpaired chunk that still fits
    std::stable_sort(ch1.begin(), ch1.end(), [](const RadChunk& p, const RadChunk& q) { return p.count > q.count; });
    std::vector<char> used(ch1.size(), 0);
    std::vector<RadPack> rl;
    for (size_t i = 0; i < ch1.size(); i++) {
        if (used[i]) continue;
        used[i] = 1;
        RadPack pk{};
        pk.c[0] = ch1[i];
        pk.c[1] = RadChunk{ch1[i].ks, ch1[i].kappa, ch1[i].first, 0};
        for (size_t j = i + 1; j < ch1.size(); j++)
            if (!used[j] && ch1[i].count + ch1[j].count <= FLANE) {
                used[j] = 1;
                pk.c[1] = ch1[j];
                break;
            }
        rl.push_back(pk);
    }
    // the pair terms' coefficients (cA, cB) = (-c tau A1, c tau A2), from their double-float words
    std::vector<float4> cdf(B.pterm.size());
    if (!cdf.empty())
        CUDA_TRY(cudaMemcpy(cdf.data(), op->cab_df, sizeof(float4) * cdf.size(), cudaMemcpyDeviceToHost));
    // per channel: its (partner, multipole, coefficients of U, V, U', V') terms
    struct Use { int b, l; double c[4]; };
    std::vector<std::vector<Use>> uses(nch);
    for (size_t p = 0; p < B.pa.size(); p++) {
        const int a = B.pa[p], b = B.pb[p];
        for (int q = B.pterm_start[p]; q < B.pterm_start[p + 1]; q++) {
            const double cA = (double)cdf[q].x + (double)cdf[q].y, cB = (double)cdf[q].z + (double)cdf[q].w;
            const double ka = B.kap[a], kb = B.kap[b];
            uses[a].push_back(Use{b, B.pterm[q].l, {-cA, -cA * ka, -cB, -cB * ka}});
            uses[b].push_back(Use{a, B.pterm[q].l, {cB, cB * kb, cA, cA * kb}});
        }
    }
    std::vector<int> tms(B.tmu.begin(), B.tmu.end());
    std::sort(tms.begin(), tms.end());
    tms.erase(std::unique(tms.begin(), tms.end()), tms.end());
    auto lparity = [](int k) { return (k > 0 ? k : -k - 1) & 1; };
    std::vector<FactSub> subs;
    std::vector<int> ioff;
    std::vector<float4> icoef;
    for (int tm : tms) {
        std::vector<int> chs;
        for (int a = 0; a < nch; a++)
            if (B.tmu[a] == tm) chs.push_back(a);
        std::stable_sort(chs.begin(), chs.end(), [&](int p, int q) {
            const int kp = B.kap[p], kq = B.kap[q];
            if (lparity(kp) != lparity(kq)) return lparity(kp) < lparity(kq);
            if (std::abs(kp) != std::abs(kq)) return std::abs(kp) < std::abs(kq);
            return kp < kq;
        });
        for (size_t s0 = 0; s0 < chs.size(); s0 += FSG) {
            FactSub g{};
            g.first = (int)ioff.size();
            std::map<std::pair<int, int>, std::array<float4, FSG>> items;   // (partner, l), ordered
            for (int j = 0; j < FSG; j++) {
                g.out[j] = s0 + j < chs.size() ? chs[s0 + j] : -1;
                if (g.out[j] < 0) continue;
                for (const Use& u : uses[g.out[j]]) {
                    auto key = std::make_pair(u.b, u.l);
                    auto it = items.find(key);
                    if (it == items.end()) {
                        std::array<float4, FSG> z;
                        z.fill(make_float4(0.f, 0.f, 0.f, 0.f));
                        it = items.emplace(key, z).first;
                    }
                    it->second[j] = make_float4((float)u.c[0], (float)u.c[1], (float)u.c[2], (float)u.c[3]);
                }
            }
            for (auto& kv : items) {
                ioff.push_back(kv.first.first * L + kv.first.second);
                for (int j = 0; j < FSG; j++) icoef.push_back(kv.second[j]);
            }
            g.count = (int)ioff.size() - g.first;
            subs.push_back(g);
        }
    }
    // heaviest subgroups first, so the long blocks start in the first wave
    std::stable_sort(subs.begin(), subs.end(), [](const FactSub& p, const FactSub& q) { return p.count > q.count; });
    if (ioff.empty()) { ioff.push_back(0); icoef.assign(FSG, make_float4(0.f, 0.f, 0.f, 0.f)); }
    dirac_status e = upload(op, &op->rad_lanes, rl);
    if (!e) e = upload(op, &op->fsub, subs);
    if (!e) e = upload(op, &op->fitem_off, ioff);
    if (!e) e = upload(op, &op->fitem_coef, icoef);
    if (e) return e;
    op->nrad_lanes = (int)rl.size();
    op->nfsub = (int)subs.size();
    op->fsub_max = subs.empty() ? 1 : std::max(1, subs[0].count);   // sorted by decreasing count
    CUDA_TRY(fact_sub_prepare(op->fsub_max));
    return DIRAC_OK;
}

extern "C" dirac_status dirac_op_set_factorised(dirac_op* op, int enable)
{
    if (!op || enable < 0 || enable > 2 ||
        (enable && (op->opts.precision != 2 || op->ov.bd != 13 || !op->cab_df || !op->S32T))) {
        set_error("dirac_op_set_factorised: needs precision 2, order-7 splines and a mode 0, 1 or 2");
        return DIRAC_E_ARG;
    }
    if (enable == 2 && !op->rad_chunks) {
        // kappa groups of the kappa-sorted channel order, in chunks of at most FCOL channels
        std::vector<int> ks(op->ov.nch), ordv(op->ov.nch), kap(op->ov.nch);
        CUDA_TRY(cudaMemcpy(ordv.data(), op->ov.prec_order, sizeof(int) * ordv.size(), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(ks.data(), op->ov.ch_kslot, sizeof(int) * ks.size(), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(kap.data(), op->ov.ch_kappa, sizeof(int) * kap.size(), cudaMemcpyDeviceToHost));
        std::vector<RadChunk> rc;
        for (int i = 0; i < op->ov.nch;) {
            int j = i;
            while (j < op->ov.nch && ks[ordv[j]] == ks[ordv[i]] && j - i < FCOL) j++;
            rc.push_back(RadChunk{ks[ordv[i]], kap[ordv[i]], i, j - i});
            i = j;
        }
        dirac_status e = upload(op, &op->rad_chunks, rc);
        if (e) return e;
        op->nrad = (int)rc.size();
    }
    if (enable == 1 && !op->fsub) {
        dirac_status e = fact_sub_setup(op);
        if (e) return e;
        // the G hi words as plain floats, written by every later assembly of each buffer set
        const size_t gsz = (size_t)op->pv.L * 4 * op->ov.n1 * op->ov.bd * 4;
        for (int c = 0; c < 2; c++)
            if (op->aset[c].Gdf && !op->aset[c].Ghi && (e = dev_alloc(op, &op->aset[c].Ghi, gsz))) return e;
        op->Ghi = op->aset[op->acur].Ghi;
    }
    if (enable && !op->Zf) {
        // products of two radial tiles (the subgroup form forms tile t + 1 while it combines tile t)
        dirac_status e = dev_alloc(op, &op->Zf, (size_t)2 * op->ov.nch * op->pv.L * 4 * FTR * 2);
        if (e) return e;
    }
    op->fact32 = enable;
    op->config_gen++;   // captured graphs hold the other apply
    return DIRAC_OK;
}

extern "C" int dirac_op_get_schedule(const dirac_op* op, int complex64)
{
    if (!op) return -1;
    return complex64 ? op->prec_sched32 : op->prec_sched64;
}

// make buffer set c the current one (the pointers every precision-2 kernel reads)
static void select_set(dirac_op* op, int c)
{
    if (c == op->acur) return;
    const AsmSet& a = op->aset[c];
    op->t_eval = a.t_eval;
    op->s = a.s;
    op->Gdf = a.Gdf;
    op->Ghi = a.Ghi;
    op->Kdf = a.Kdf;
    op->KTdf = a.KTdf;
    op->Wh = a.Wh;
    op->Wl = a.Wl;
    op->k32.W = a.Wh;
    op->acur = c;
    op->config_gen++;   // captured graphs hold the old pointers
}

extern "C" dirac_status dirac_op_set_residual_mode(dirac_op* op, int mode)
{
    if (!op || mode < 0 || mode > 2) {
        set_error("dirac_op_set_residual_mode: bad argument (mode 0, 1 or 2)");
        return DIRAC_E_ARG;
    }
    if (mode != op->resid_mode) {
        op->resid_mode = mode;
        op->config_gen++;   // captured graphs hold the other launch sequence
    }
    return DIRAC_OK;
}

extern "C" dirac_status dirac_op_set_overlap(dirac_op* op, int enable)
{
    if (!op || (enable && op->opts.precision != 2)) {
        set_error("dirac_op_set_overlap: bad argument (the overlapped assembly needs precision 2)");
        return DIRAC_E_ARG;
    }
    if (enable && !op->aset[1].Wh) {
        size_t be = (size_t)op->ov.n1 * op->ov.bd * 4;
        AsmSet a;
        dirac_status e;
        if ((e = dev_alloc(op, &a.t_eval, 1)) || (e = dev_alloc(op, &a.s, (size_t)op->pv.L * 3)) ||
            (e = dev_alloc(op, &a.Gdf, (size_t)op->pv.L * 4 * be)) ||
            (!op->asm_chunks && (e = dev_alloc(op, &a.Kdf, (size_t)std::max(op->ov.nkeys, 1) * be))) ||
            (!op->asm_chunks && (e = dev_alloc(op, &a.KTdf, (size_t)std::max(op->ov.nkeys, 1) * be))) ||
            (e = dev_alloc(op, &a.Wh, (size_t)std::max<int64_t>(op->npairs, 1) * be)) ||
            (e = dev_alloc(op, &a.Wl, (size_t)std::max<int64_t>(op->npairs, 1) * be)))
            return e;
        CUDA_TRY(cudaStreamCreateWithFlags(&op->st_asm, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&op->ev_res, cudaEventDisableTiming));
        for (int i = 0; i < 2; i++) {
            CUDA_TRY(cudaEventCreateWithFlags(&op->ev_asm[i], cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&op->ev_use[i], cudaEventDisableTiming));
        }
        if (op->aset[0].Ghi && (e = dev_alloc(op, &a.Ghi, (size_t)op->pv.L * 4 * be))) return e;
        op->aset[1] = a;
    }
    op->overlap = enable != 0;
    return DIRAC_OK;
}

extern "C" dirac_status dirac_step(dirac_op* op, void* psi_dev, void* hist_dev, int* n_hist, int n_steps,
                                   double t_start, int* iters_out, double* resid_out)
{
    if (!op || !psi_dev || n_steps < 0) { set_error("dirac_step: bad argument"); return DIRAC_E_ARG; }
    int64_t n = op->n;
    double2* psi = (double2*)psi_dev;
    const dirac_solver_opts& o = op->opts;
    const bool learned = o.guess == 2 && op->net;
    const int hmax = learned ? 3 : 2;   // history entries kept (the network reads three past states)
    double2* h1 = hist_dev ? (double2*)hist_dev : nullptr;
    double2* h2 = hist_dev ? (double2*)hist_dev + n : nullptr;
    double2* h3 = (hist_dev && learned) ? (double2*)hist_dev + 2 * n : nullptr;
    int nh = (hist_dev && n_hist) ? std::max(0, std::min(hmax, *n_hist)) : 0;
    int npv = op->nparts_vec;
    Krylov& K = op->k64;
    dirac_status result = DIRAC_OK;
    // overlapped assembly: step s + 1's coupling values are assembled on st_asm into the other buffer
    // set while step s solves; ev_asm[c] marks set c assembled, ev_use[c] the end of its last use
    const bool ovl = op->overlap && o.precision == 2 && op->aset[1].Wh;
    const double t_off = o.time_eval ? o.dt : 0.5 * o.dt;
    for (int step = 0; step < n_steps; step++) {
        if (!ovl || step == 0) {
            if (ovl) CUDA_TRY(cudaStreamWaitEvent(op->st, op->ev_asm[op->acur], 0));   // a pending fill of this set
            k_set_step_time<<<1, 1, 0, op->st>>>(op->t_eval, t_start, step, o.dt, t_off);
            op->launches++;
            launch_assemble(op);
        } else {
            CUDA_TRY(cudaStreamWaitEvent(op->st, op->ev_asm[op->acur], 0));
        }
        // the next step's assembly starts once this step's first residual pass is done, so that it
        // runs beside the memory- and latency-bound inner solve rather than the FP32-bound residual
        bool next_launched = !(ovl && step + 1 < n_steps);
        auto launch_next = [&]() -> dirac_status {
            if (next_launched) return DIRAC_OK;
            next_launched = true;
            const int nx = 1 - op->acur;
            CUDA_TRY(cudaEventRecord(op->ev_res, op->st));
            CUDA_TRY(cudaStreamWaitEvent(op->st_asm, op->ev_res, 0));
            CUDA_TRY(cudaStreamWaitEvent(op->st_asm, op->ev_use[nx], 0));
            k_set_step_time<<<1, 1, 0, op->st_asm>>>(op->aset[nx].t_eval, t_start, step + 1, o.dt, t_off);
            op->launches++;
            launch_assemble_set(op, op->st_asm, op->aset[nx]);
            CUDA_TRY(cudaEventRecord(op->ev_asm[nx], op->st_asm));
            return DIRAC_OK;
        };
        // b = A_- psi, ||b||^2 (precision 2 forms them inside the residual passes)
        if (o.precision == 0) {
            apply_accurate(op, -1, psi, K.b, nullptr, op->part_n);
            finish(op, K.ks, 0, op->nparts_apply, nullptr, op->part_n, o.max_iter);
        } else {
            rhs_accurate(op, psi);
        }
        // initial guess (timed as its own phase when learned, else with the vector kernels)
        {
            double2* x = (double2*)K.x;
            if (learned && nh >= 3) {
                PhaseScope pg(op, DIRAC_PHASE_GUESS, 0);   // guess_into counts its launches
                dirac_status ge = guess_into(op, psi, h1, h2, h3, t_start, step, x, nullptr, op->st, nullptr);
                if (ge) return ge;
            } else {
                PhaseScope ps(op, DIRAC_PHASE_VECTOR, 1);
                k_extrapolate<<<npv, 256, 0, op->st>>>(n, o.guess >= 1 ? std::min(nh, 2) : 0, psi, h1, h2, x);
            }
        }
        KState hs{};
        int total_it = 0;
        dirac_status e;
        if (o.precision == 0) {
            e = solve(op, K, o.max_iter, hs, &total_it, true);
            if (e) return e;
        } else {
            // iterative refinement: r = b - A x in FP64, A d = r / ||r|| by FP32 BiCGSTAB, x += ||r|| d
            Krylov& I = op->k32;
            int outer = 0;
            for (;;) {
                // true residual r = b - A x accurate to double precision; done when ||r|| <= tol ||b||
                residual_accurate(op, psi);
                e = launch_next();
                if (e) return e;
                e = read_state(op, K, hs);
                if (e) return e;
                if (hs.done || hs.status) break;
                if (outer++ >= o.max_outer) { hs.status = 4; break; }
                {
                    PhaseScope ps(op, DIRAC_PHASE_VECTOR, 2);
                    k_to_float_scaled<<<npv, 256, 0, op->st>>>(n, (const double2*)K.r, K.ks, (float2*)I.b);
                    k_zero32<<<npv, 256, 0, op->st>>>(n, (float2*)I.x);
                }
                KState hi{};
                int its = 0;
                e = solve(op, I, o.max_iter, hi, &its, false);
                if (e) return e;
                total_it += its;
                if (hi.status && hi.status != 4) { hs.status = hi.status; break; }
                PhaseScope ps(op, DIRAC_PHASE_VECTOR, 1);
                k_add_float_scaled<<<npv, 256, 0, op->st>>>(n, (const float2*)I.x, K.ks, (double2*)K.x);
            }
        }
        double res = std::sqrt(hs.rnorm2 / (hs.bnorm2 > 0 ? hs.bnorm2 : 1.0));
        if (iters_out) iters_out[step] = total_it;
        if (resid_out) resid_out[step] = res;
        // history shift and accept the iterate (also on failure, as documented)
        {
            PhaseScope ps(op, DIRAC_PHASE_VECTOR,
                          1 + (h1 ? 1 : 0) + (h2 && nh >= 1 ? 1 : 0) + (h3 && nh >= 2 ? 1 : 0));
            if (h1) {
                if (h3 && nh >= 2) k_copy64<<<npv, 256, 0, op->st>>>(n, h2, h3);
                if (h2 && nh >= 1) k_copy64<<<npv, 256, 0, op->st>>>(n, h1, h2);
                k_copy64<<<npv, 256, 0, op->st>>>(n, psi, h1);
                nh = std::min(hmax, nh + 1);
            }
            k_copy64<<<npv, 256, 0, op->st>>>(n, (const double2*)K.x, psi);
        }
        if (ovl) {
            CUDA_TRY(cudaEventRecord(op->ev_use[op->acur], op->st));
            if (step + 1 < n_steps) select_set(op, 1 - op->acur);
        }
        e = check_launch("dirac_step");
        if (e) return e;
        if (hs.status) {
            result = (dirac_status)hs.status;
            set_error("dirac_step: step " + std::to_string(step) + " failed with status " + std::to_string(hs.status) +
                      " (residual " + std::to_string(res) + ")");
            break;
        }
    }
    if (n_hist) *n_hist = nh;
    CUDA_TRY(cudaStreamSynchronize(op->st));
    if (op->st_asm) CUDA_TRY(cudaStreamSynchronize(op->st_asm));
    collect_phases(op);
    dirac_status de = check_dev_err(op, "dirac_step");
    if (de) return de;
    return result;
}

__global__ void k_observe(OpView A, const double2* __restrict__ x, const double2* __restrict__ g, int gch,
                          double2* part_a, double2* part_c)
{
    // per thread (channel, slot): (S x), (H0 x); partial x^H S x, x^H H0 x and g^T S x_gch
    int ch = blockIdx.y, r = blockIdx.x * blockDim.x + threadIdx.x;
    double xs = 0, xh = 0;
    double2 gp = make_double2(0, 0);
    if (r < A.n1) {
        const double2* xa = x + (int64_t)ch * 2 * A.n1;
        int ks = A.ch_kslot[ch];
        const double* Sk = A.S + ((int64_t)ks * A.n1 + r) * A.bd * 4;
        const double* Hk = A.H + ((int64_t)ks * A.n1 + r) * A.bd * 4;
        for (int t = 0; t < 2; t++) {
            double2 sx = make_double2(0, 0), hx = make_double2(0, 0);
            for (int d = 0; d < A.bd; d++) {
                int rr = r + d - A.half;
                if (rr < 0 || rr >= A.n1) continue;
                for (int u = 0; u < 2; u++) {
                    double2 xv = xa[2 * rr + u];
                    double sv = Sk[d * 4 + t * 2 + u], hv = Hk[d * 4 + t * 2 + u];
                    sx.x += sv * xv.x; sx.y += sv * xv.y;
                    hx.x += hv * xv.x; hx.y += hv * xv.y;
                }
            }
            double2 xi = xa[2 * r + t];
            xs += xi.x * sx.x + xi.y * sx.y;
            xh += xi.x * hx.x + xi.y * hx.y;
            if (ch == gch) {
                double2 gv = g[2 * r + t];  // real eigenvector (imaginary part zero)
                gp.x += gv.x * sx.x;
                gp.y += gv.x * sx.y;
            }
        }
    }
    int64_t slot = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    block_reduce_store(make_double2(xs, xh), 0.0, part_a, nullptr, slot);
    block_reduce_store(gp, 0.0, part_c, nullptr, slot);
}

extern "C" dirac_status dirac_observables(dirac_op* op, const void* psi_dev, double* out, int n_out)
{
    if (!op || !psi_dev || !out || n_out < 1 || n_out > 4) { set_error("dirac_observables: bad argument"); return DIRAC_E_ARG; }
    dim3 grid(grid_for(op->ov.n1, 128), op->ov.nch);
    k_observe<<<grid, 128, 0, op->st>>>(op->ov, (const double2*)psi_dev, op->psi0_g, op->ground_ch, op->part_d,
                                         op->part_d2);
    op->launches++;
    dirac_status e = check_launch("dirac_observables");
    if (e) return e;
    int np = op->nparts_apply;
    std::vector<double2> a(np), c(np);
    CUDA_TRY(cudaMemcpyAsync(a.data(), op->part_d, sizeof(double2) * np, cudaMemcpyDeviceToHost, op->st));
    CUDA_TRY(cudaMemcpyAsync(c.data(), op->part_d2, sizeof(double2) * np, cudaMemcpyDeviceToHost, op->st));
    CUDA_TRY(cudaStreamSynchronize(op->st));
    double ns = 0, nh = 0, gx = 0, gy = 0;
    for (int i = 0; i < np; i++) { ns += a[i].x; nh += a[i].y; gx += c[i].x; gy += c[i].y; }
    double vals[4] = {ns, nh, gx * gx + gy * gy, 0.0};
    if (n_out >= 4) {
        e = bound_population(op, (const double2*)psi_dev, &vals[3]);
        if (e) return e;
    }
    for (int i = 0; i < n_out; i++) out[i] = vals[i];
    return DIRAC_OK;
}

// ---------------------------------------------------------------------------------------------
// Observables with library-static scratch (no allocation in the call).
//
// Some callers cannot allocate GPU memory when they need the observables: real-time or monitoring
// threads that must not hit the implicit device synchronisation of cudaMalloc/cudaFree, and hosts
// that fix the process's device footprint after setup.  dirac_observables_static serves them: its
// block partials and the final sums live in the file-scope array below, which the driver places
// in device memory when it loads this module on a device (at the module's first use there, e.g. in
// dirac_operator_setup) and which that GPU holds until the process exits.  The call itself calls no
// cudaMalloc, cudaFree or other allocating routine, on the device or the host.
// ---------------------------------------------------------------------------------------------
static __device__ __align__(256) double2 g_obs_scratch[2 * DIRAC_STATIC_MAX_PARTIALS + 2];

namespace dg {

// device address of g_obs_scratch, looked up once per device with that device current (host code
// must not use the symbol itself as a device address: in host code it names a host-side stand-in).
// dirac_operator_setup looks it up, so the observables call does no set-up of its own.  The address
// is kept for the life of the process; after a cudaDeviceReset the module is loaded again, possibly
// elsewhere, so the library must not be used across a device reset.
static std::mutex g_obs_mutex;
static void* g_obs_addr[64] = {nullptr};

dirac_status obs_scratch_address(int device, double2** out)
{
    if (device < 0 || device >= 64) { set_error("dirac_observables_static: device index beyond 63"); return DIRAC_E_ARG; }
    std::lock_guard<std::mutex> lock(g_obs_mutex);
    if (!g_obs_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_obs_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("dirac_observables_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return DIRAC_E_CUDA;
        }
        g_obs_addr[device] = p;
    }
    *out = (double2*)g_obs_addr[device];
    return DIRAC_OK;
}

// fixed-order sum of the block partials into out[0] = (sum a.x, sum a.y), out[1] = (sum c.x, sum c.y)
__global__ void k_obs_sum(int np, const double2* part_a, const double2* part_c, double2* out)
{
    __shared__ double s[4][1024];
    int t = threadIdx.x;
    double v[4] = {0, 0, 0, 0};
    for (int i = t; i < np; i += blockDim.x) {
        v[0] += part_a[i].x; v[1] += part_a[i].y;
        v[2] += part_c[i].x; v[3] += part_c[i].y;
    }
    for (int k = 0; k < 4; k++) s[k][t] = v[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int k = 0; k < 4; k++) s[k][t] += s[k][t + w];
        __syncthreads();
    }
    if (t == 0) {
        out[0] = make_double2(s[0][0], s[1][0]);
        out[1] = make_double2(s[2][0], s[3][0]);
    }
}

}  // namespace dg

extern "C" dirac_status dirac_observables_static(dirac_op* op, const void* psi_dev, double* out, int n_out)
{
    if (!op || !psi_dev || !out || n_out < 1 || n_out > 3) {
        set_error("dirac_observables_static: bad argument");
        return DIRAC_E_ARG;
    }
    int np = op->nparts_apply;
    if (np > DIRAC_STATIC_MAX_PARTIALS) {
        set_error("dirac_observables_static: " + std::to_string(np) + " block partials (channels x ceil((N+1)/128)) "
                  "exceed the static scratch of " + std::to_string(DIRAC_STATIC_MAX_PARTIALS) +
                  "; use dirac_observables");
        return DIRAC_E_ARG;
    }
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev != op->device) { set_error("dirac_observables_static: current device differs from the op's"); return DIRAC_E_STATE; }
    // the call copies its sums to the host and synchronises the op's stream, which a stream capture
    // does not allow: refuse before anything is enqueued, so the caller's capture stays valid
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(op->st, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
        set_error("dirac_observables_static: the op's stream is being captured (the call synchronises it)");
        return DIRAC_E_STATE;
    }
    double2* scratch = nullptr;
    dirac_status e = obs_scratch_address(dev, &scratch);
    if (e) return e;
    // layout: [0, np) partials of (x^H S x, x^H H0 x); [M, M + np) partials of g^T S x; 2M, 2M+1: sums.
    // Every slot read below is written earlier in this call, so nothing has to be cleared.
    double2* pa = scratch;
    double2* pc = scratch + DIRAC_STATIC_MAX_PARTIALS;
    double2* sums = scratch + 2 * DIRAC_STATIC_MAX_PARTIALS;
    dim3 grid(grid_for(op->ov.n1, 128), op->ov.nch);
    k_observe<<<grid, 128, 0, op->st>>>(op->ov, (const double2*)psi_dev, op->psi0_g, op->ground_ch, pa, pc);
    k_obs_sum<<<1, 1024, 0, op->st>>>(np, pa, pc, sums);
    op->launches += 2;
    e = check_launch("dirac_observables_static");
    if (e) return e;
    double2 h[2];
    CUDA_TRY(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, op->st));
    CUDA_TRY(cudaStreamSynchronize(op->st));
    double vals[3] = {h[0].x, h[0].y, h[1].x * h[1].x + h[1].y * h[1].y};
    for (int i = 0; i < n_out; i++) out[i] = vals[i];
    return DIRAC_OK;
}
