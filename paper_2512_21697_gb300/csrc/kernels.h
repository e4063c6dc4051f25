// kernels.h -- kernel declarations and the block reduction helper shared by the .cu files.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device.h"

namespace dg {

// Sum a (complex, real) pair over the block in a fixed order and store the block's partials.
// Every thread of the block must call it.  Block size must be a multiple of 32, <= 1024.  A part
// whose output is NULL is not reduced (FP64 adds are scarce on this part: a norm-only reduction
// costs a third of a full one); the parts kept are summed in the same order either way.
__device__ __forceinline__ void block_reduce_store(double2 d, double n, double2* out_d, double* out_n, int64_t slot)
{
    __shared__ double2 wd[32];
    __shared__ double wn[32];
    const bool want_d = out_d != nullptr, want_n = out_n != nullptr;   // uniform over the block
    for (int off = 16; off > 0; off >>= 1) {
        if (want_d) {
            d.x += __shfl_down_sync(0xffffffffu, d.x, off);
            d.y += __shfl_down_sync(0xffffffffu, d.y, off);
        }
        if (want_n) n += __shfl_down_sync(0xffffffffu, n, off);
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        if (want_d) wd[warp] = d;
        if (want_n) wn[warp] = n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 sd = make_double2(0, 0);
        double sn = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            if (want_d) { sd.x += wd[w].x; sd.y += wd[w].y; }
            if (want_n) sn += wn[w];
        }
        if (want_d) out_d[slot] = sd;
        if (want_n) out_n[slot] = sn;
    }
    __syncthreads();
}

__global__ void k_time_factors(PulseView P, const double* t_eval, double* s);
__global__ void k_field_combine(PulseView P, int block_elems, const double* s, double* G);
__global__ void k_build_K(OpView A, int block_elems, const double* G, double* K);
__global__ void k_assemble64(OpView A, const double* K, double* W, float* W32);
// y = A_sign x (+ epilogues) in precision T, 128 threads per block, grid (channels, slots / 128)
template <class T>
void launch_apply_t(dim3 grid, cudaStream_t st, const OpView& A, const T* S, const T* H, int sign, const void* x,
                    const T* W, void* y, const void* bsub, const void* dv, double2* pdot, double* pnrm,
                    const KState* skip);
// z = M^-1 (prologue-formed vector) in precision T, 32 threads (channels) per block
template <class T>
void launch_precond_t(int blocks, cudaStream_t st, const OpView& A, const void* U, const void* L, const void* Dinv,
                      int mode, const KState* ks, const void* r, const void* v, void* io, void* z, double* pn);
// lane-per-channel preconditioner (band width 13), one warp per same-kappa channel group
template <class T>
void launch_precond_lanes_t(int nwarps, cudaStream_t st, const OpView& A, const void* Urow, const void* L,
                            const void* Dinv, const int* wks, const int* wfirst, const int* wcnt, int mode,
                            const KState* ks, const void* r, const void* v, void* io, void* z, double* pn);
template <class T>
void launch_update_xr_t(int blocks, cudaStream_t st, int64_t n, const KState* ks, void* x, void* r, const void* ph,
                        const void* sh, const void* s, const void* t, const void* rh, double2* pd, double* pn);
__global__ void k_to_float_scaled(int64_t n, const double2* a, const KState* st, float2* b);
__global__ void k_add_float_scaled(int64_t n, const float2* d, const KState* st, double2* x);
__global__ void k_copy32(int64_t n, const float2* a, float2* b);
// double-float path (precision 2)
__global__ void k_split_vec(int64_t n, const double2* __restrict__ x, float4* __restrict__ xd);
__global__ void k_field_combine_df(PulseView P, int block_elems, const double* s, float2* G, float* Gh);
__global__ void k_build_K_df(OpView A, int block_elems, const float2* G, float2* K, float2* KT);
void launch_assemble_df(dim3 grid, cudaStream_t st, const OpView& A, const float2* K, const float2* KT, const float4* cab, float* Wh,
                        float* Wl);
// grouped assembly: grid (positions / 128, chunks); gpair/gcoef in group order, ASM_MAX_NL
// (cA hi, cA lo, cB hi, cB lo) per pair
void launch_assemble_grp_df(cudaStream_t st, const OpView& A, const AsmChunk* chunks, int nchunks, const int* gpair,
                            const float4* gcoef, const float2* G, float* Wh, float* Wl);
// type-major split vectors ([channel][DKB type][slot]) of the owner/gather residual passes
__global__ void k_split_uv3(int64_t n, int n1, const double2* psi, const double2* x, float4* u, float4* v,
                            float2* psi32);
__global__ void k_split_uv(int64_t n, const double2* __restrict__ psi, const double2* __restrict__ x,
                           float4* __restrict__ u, float4* __restrict__ v);
void launch_residual_df(dim3 grid, cudaStream_t st, const OpView& A, const float2* S, const float2* Ht, const float4* u,
                        const float4* v, const float* Wh, const float* Wl, double2* r, double* pr, double* pb);
void launch_apply_df(dim3 grid, cudaStream_t st, const OpView& A, const float2* S, const float2* Ht, int sign,
                     const float4* x, const float* Wh, const float* Wl, double2* y, const double2* bsub, double* pn);
__global__ void k_zero32(int64_t n, float2* a);
__global__ void k_copy64(int64_t n, const double2* a, double2* b);
__global__ void k_zero64(int64_t n, double2* a);
__global__ void k_lincomb64(int64_t n, double c0, const double2* a, double c1, const double2* b, double c2,
                            const double2* c, double2* x);
__global__ void k_finish64(int what, KState* st, int np, const double2* pd, const double* pn, const double2* pd2,
                           const double* pn2, int max_iter);
__global__ void k_set_time(double* t_eval, double t);
__global__ void k_bnorm_if(KState* st, int* flag, int np, const double* pn);
__global__ void k_set_int(int* p, int v);
__global__ void k_set_step_time(double* t_eval, double t_start, int step, double dt, double t_off);
// evaluation time of step `step`: (t_start + step dt) + t_off, each operation rounded separately
// (no contraction), so the host-driven and the graph-driven loops agree to the last bit
__device__ __forceinline__ double step_time(double t_start, int step, double dt, double t_off)
{
    return __dadd_rn(__dadd_rn(t_start, __dmul_rn((double)step, dt)), t_off);
}

// initial guess from the last states, polynomial extrapolation in time: 3 psi - 3 h1 + h2 (two
// past states), 2 psi - h1 (one), psi (none); explicit rounding so both step loops agree bitwise
__device__ __forceinline__ double extrapolate(int nh, double p, double a, double b)
{
    if (nh >= 2) return __dadd_rn(__dmul_rn(3.0, __dsub_rn(p, a)), b);
    if (nh == 1) return __dsub_rn(__dmul_rn(2.0, p), a);
    return p;
}
__global__ void k_extrapolate(int64_t n, int nh, const double2* psi, const double2* h1, const double2* h2, double2* x);

// the learned guess's six field factors at time t (the separable carriers of the sin^2 pulse)
__device__ __forceinline__ void guess_field_at(const PulseView& P, double t, float* f)
{
    double tt = t - P.t0;
    bool on = tt >= 0 && tt <= P.T;
    for (int c = 0; c < 3; c++) {
        f[2 * c] = on ? (float)(P.amp * P.wt[c] * sin(P.w[c] * tt)) : 0.f;
        f[2 * c + 1] = on ? (float)(P.amp * P.wt[c] * cos(P.w[c] * tt)) : 0.f;
    }
}
// time of step `step` + 1 from a start time, explicitly rounded (host loop and graph agree)
__device__ __forceinline__ double next_time(double t_start, int step, double dt)
{
    return __dadd_rn(t_start, __dmul_rn((double)(step + 1), dt));
}

// warp-per-channel preconditioner with shared-memory staging (band width 13)
template <class T> size_t precond_sm_smem(int n1);
template <class T> cudaError_t precond_sm_prepare(int n1);
template <class T> int precond_sm_blocks(int nch);
template <class T>
void launch_precond_sm_t(cudaStream_t st, const OpView& A, const void* U, const void* L, const void* Dinv, int mode,
                         const KState* ks, const void* r, const void* v, void* io, void* z, double* pn);

// rotated-lane warp-per-channel preconditioner (band width 13): factor chunks only in shared memory
template <class T> cudaError_t precond_rot_prepare();
template <class T> int precond_rot_blocks(int nch);
template <class T>
void launch_precond_rot_t(cudaStream_t st, const OpView& A, const void* U, const void* L, const void* Dinv, int mode,
                          const KState* ks, const void* r, const void* v, void* io, void* z, double* pn);

// bounded-wait self-test: one block waits `limit` cycles on an mbarrier nothing completes
cudaError_t launch_wait_selftest(cudaStream_t st, long long limit, int* err);

// factorised complex64 apply (coupling values never stored): radial + angular pass per tile, in the
// per-channel form (partials: one per tile and channel) or the subgroup form (one per tile and
// subgroup; ST, HT the FP32 diagonal bands with the rows innermost)
int fact_tile();
void launch_fact32_chan(cudaStream_t st, const OpView& A, const RadChunk* rc, int nrc, const float2* G, int L,
                        const float* S, const float* H, int sign, const void* x, float2* Z, const float4* cab,
                        void* y, const void* bsub, const void* dv, double2* pdot, double* pnrm, const KState* skip);
cudaError_t fact_sub_prepare(int max_items);   // dynamic shared-memory limits (once per device)
void launch_fact32_sub(cudaStream_t st, const OpView& A, const RadPack* rl, int nrl, const FactSub* subs, int nsub,
                       int max_items, const int* item_off, const float4* item_coef, const float* Gh, int L,
                       const float* ST, const float* HT, int sign, const void* x, float2* Z, void* y,
                       const void* bsub, const void* dv, double2* pdot, double* pnrm, const KState* skip);

// learned-guess network forward on the fifth-generation tensor cores (tcgen05, TMEM accumulators)
size_t guess_forward_tc05_smem();
int64_t guess_tc05_packed();
int guess_tc05_rows();
cudaError_t guess_tc05_prepare();
void launch_pack_tc05(cudaStream_t st, const __nv_bfloat16* wb, __nv_bfloat16* wt);
void launch_guess_forward_tc05(cudaStream_t st, int64_t M, const float* X, const __nv_bfloat16* wt,
                               const float* b1, const float* b2, const float* b3, const float* b4, float* out,
                               const int* gate, int* err);

// complex64 apply with each coupling block read once (owner pass + gather pass, bd = 13)
size_t apply_own32_smem();
int apply_own_tile();
int apply_own_nout();
bool apply_own_supported(const OpView& A);
cudaError_t apply_own32_prepare();
size_t residual_own_df_smem();
// the double-float residual's owner pass reads one offset byte per accumulator (df_fma_off):
// launch_residual_offsets forms them from the u-window sums US (residual_us_floats, written here), the
// static envelopes E, Ew ([L][4][n1] floats), the grouped assembly's chunks and coefficients and
// the time factors s, into sig (npairs x tiles x residual_sig_bytes() bytes)
void launch_residual_offsets(cudaStream_t st, const OpView& A, const AsmChunk* chunks, int nchunks, const int* gpair,
                             const float4* gcoef, const double* s, const float* E, const float* Ew, float* US,
                             unsigned char* sig, const float4* u);
// offsets: the fixed-binade accumulators (sig from launch_residual_offsets), else the Dot2 form (sig unused)
void launch_residual_owner_df(cudaStream_t st, const OpView& A, bool offsets, const unsigned char* sig,
                              const float4* u, const float2* psi32, const float* Wh, const float* Wl, double2* r,
                              float2* b, float4* part_r, float4* part_b, const int* need_b, int* err);
int residual_sig_bytes();
size_t residual_us_floats(int nch, int n1);   // size of the u-window-sum buffer US (zeroed once)
// S, Ht: the diagonal bands with the rows innermost ([kappa slot][d][row][entry] float2)
void launch_residual_gather_df(cudaStream_t st, const OpView& A, const float2* S, const float2* Ht, const float4* u,
                               const float4* v, const float2* psi32, double2* r, const float2* b,
                               const float4* part_r, const float4* part_b, const int* need_b, double* pn_r,
                               double* pn_b);
// S, H: the FP32 diagonal bands with the rows innermost ([kappa slot][d][row][entry])
void launch_apply_own32(cudaStream_t st, const OpView& A, const float* S, const float* H, int sign, const void* x,
                        const float* W, void* y, float4* part, const void* bsub, const void* dv, double2* pdot,
                        double* pnrm, const KState* skip, int* err);

}  // namespace dg
