// kernels.h -- kernel declarations and the block reduction helper shared by the .cu files.
#pragma once
#include <cuda_runtime.h>

#include "device.h"

namespace dg {

// Sum a (complex, real) pair over the block in a fixed order and store the block's partials.
// Every thread of the block must call it.  Block size must be a multiple of 32, <= 1024.
__device__ __forceinline__ void block_reduce_store(double2 d, double n, double2* out_d, double* out_n, int64_t slot)
{
    __shared__ double2 wd[32];
    __shared__ double wn[32];
    for (int off = 16; off > 0; off >>= 1) {
        d.x += __shfl_down_sync(0xffffffffu, d.x, off);
        d.y += __shfl_down_sync(0xffffffffu, d.y, off);
        n += __shfl_down_sync(0xffffffffu, n, off);
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { wd[warp] = d; wn[warp] = n; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 sd = make_double2(0, 0);
        double sn = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            sd.x += wd[w].x; sd.y += wd[w].y; sn += wn[w];
        }
        if (out_d) out_d[slot] = sd;
        if (out_n) out_n[slot] = sn;
    }
    __syncthreads();
}

__global__ void k_time_factors(PulseView P, const double* t_eval, double* s);
__global__ void k_field_combine(PulseView P, int block_elems, const double* s, double* G);
__global__ void k_assemble64(OpView A, const double* G, double* W, float* W32);
// y = A_sign x (+ epilogues) in precision T, 128 threads per block, grid (slots / 128, channels)
template <class T>
void launch_apply_t(dim3 grid, cudaStream_t st, const OpView& A, const T* S, const T* H, int sign, const void* x,
                    const T* W, void* y, const void* bsub, const void* dv, double2* pdot, double* pnrm,
                    const KState* skip);
// z = M^-1 (prologue-formed vector) in precision T, 32 threads (channels) per block
template <class T>
void launch_precond_t(int blocks, cudaStream_t st, const OpView& A, const void* U, const void* L, int mode,
                      const KState* ks, const void* r, const void* v, void* io, void* z, double* pn);
template <class T>
void launch_update_xr_t(int blocks, cudaStream_t st, int64_t n, const KState* ks, void* x, void* r, const void* ph,
                        const void* sh, const void* s, const void* t, const void* rh, double2* pd, double* pn);
__global__ void k_to_float_scaled(int64_t n, const double2* a, const KState* st, float2* b);
__global__ void k_add_float_scaled(int64_t n, const float2* d, const KState* st, double2* x);
__global__ void k_copy32(int64_t n, const float2* a, float2* b);
__global__ void k_zero32(int64_t n, float2* a);
__global__ void k_copy64(int64_t n, const double2* a, double2* b);
__global__ void k_zero64(int64_t n, double2* a);
__global__ void k_lincomb64(int64_t n, double c0, const double2* a, double c1, const double2* b, double c2,
                            const double2* c, double2* x);
__global__ void k_finish64(int what, KState* st, int np, const double2* pd, const double* pn, const double2* pd2,
                           const double* pn2, int max_iter);
__global__ void k_set_time(double* t_eval, double t);

}  // namespace dg
