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
__global__ void k_assemble64(OpView A, const double* G, double* W);
// y = A_sign x (+ epilogues), 128 threads per block, grid (slots / 128, channels)
void launch_apply64(dim3 grid, cudaStream_t st, const OpView& A, int sign, const double2* x, const double* W,
                    double2* y, const double2* bsub, const double2* dv, double2* pdot, double* pnrm,
                    const KState* skip);
__global__ void k_precond64(OpView A, int mode, const KState* st, const double2* __restrict__ r,
                            const double2* __restrict__ v, double2* __restrict__ io, double2* __restrict__ z,
                            double* part_nrm);
__global__ void k_update_xr64(int64_t n, KState* st, double2* x, double2* r, const double2* ph, const double2* sh,
                              const double2* s, const double2* t, const double2* rh, double2* part_dot,
                              double* part_nrm);
__global__ void k_copy64(int64_t n, const double2* a, double2* b);
__global__ void k_zero64(int64_t n, double2* a);
__global__ void k_lincomb64(int64_t n, double c0, const double2* a, double c1, const double2* b, double c2,
                            const double2* c, double2* x);
__global__ void k_finish64(int what, KState* st, int np, const double2* pd, const double* pn, const double2* pd2,
                           const double* pn2, int max_iter);
__global__ void k_set_time(double* t_eval, double t);

}  // namespace dg
