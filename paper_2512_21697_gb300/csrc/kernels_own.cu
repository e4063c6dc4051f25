// kernels_own.cu -- the complex64 operator apply A_+- x of the inner solve (Eq. solPsi with the
// coupling of Eq. fullH) with every stored coupling block read from HBM once.
//
// A coupling block W_ab (pair a < b) is used twice: W_ab x_b in the rows of channel a and W_ab^T x_a
// in the rows of channel b.  Two passes:
//   k_apply_own32:    block = (channel a, tile of TR = 116 radial rows), 288 threads.  For each
//                     pair the channel owns, a producer warp copies the TR rows of W_ab and the
//                     window of x_b the band needs into shared memory with the bulk-copy engine
//                     (cp.async.bulk into an NST-deep ring: a "full" mbarrier per stage completes on
//                     the bytes, an "empty" one when the consumers release it).  Two groups of four
//                     warps take the two products of a pair: one accumulates W_ab x_b for its row,
//                     the other forms the transposed product W_ab^T x_a restricted to those rows
//                     (TR + 2h = 128 output rows, one per thread) and stores it in the pair's
//                     partial slot; the groups swap roles from pair to pair.
//                     y_a = D x_a - sign sum W_ab x_b.
//   k_apply_gather32: block = (channel b, tile).  y_b += sign sum of the partials of the pairs b is
//                     the upper channel of (own tile, and the halo rows of the two neighbouring
//                     tiles), in a fixed order, then the BiCGSTAB epilogues (y <- bsub - y, <dv, y>,
//                     ||y||^2).
// HBM traffic per apply: the coupling values once, plus 2 x 16 B per (pair, row) of partials, i.e.
// 8 % of the values' bytes at bd = 13.  Sums are formed in a fixed order, so results are
// reproducible run to run.
//
// The refinement residual of the mixed-precision step has the same two-pass form in double-float
// arithmetic (k_residual_own_df / k_residual_gather_df): the ring holds the hi and lo words of the
// coupling values, partials are stored in double.
#include <cuda_runtime.h>

#include <cstdint>

#include "df64.cuh"
#include "device.h"
#include "kernels.h"
#include "mbar.cuh"

namespace dg {

namespace {

constexpr int NT = 128;          // threads per role: NT direct-product threads, NT transposed ones
constexpr int TR = 116;          // radial rows per tile: TR + 2h = NT transposed output rows
constexpr int NST = 2;           // bulk-copy ring depth of the complex64 pass
constexpr int BDO = 13;          // block diagonals (order-7 splines)
constexpr int HO = (BDO - 1) / 2;
constexpr int ROWF = BDO * 4;    // floats per stored row of one pair
constexpr int NOUT = TR + 2 * HO;
static_assert(NOUT == NT, "one transposed output row per thread");
constexpr int STAGE32 = TR * ROWF + NOUT * 4;   // floats per complex64 ring stage: coupling rows, x_b row window
}  // namespace

// Self-test of the bounded wait: one block waits on an mbarrier phase that nothing completes, with
// the given cycle limit, then records the time-out in *err exactly as the owner passes do (no copy
// is in flight, so the block can leave at once).
__global__ void k_wait_selftest(long long limit, int* err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    bool ok = mbar_wait(&bar, 0, limit);   // phase 0 never completes: no thread arrives
    __syncthreads();
    if (threadIdx.x == 0 && !ok) atomicExch(err, 1);
}

cudaError_t launch_wait_selftest(cudaStream_t st, long long limit, int* err)
{
    k_wait_selftest<<<1, 32, 0, st>>>(limit, err);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(2 * NT + 32) k_apply_own32(OpView A, const float* __restrict__ S,
                                                             const float* __restrict__ H, int sign,
                                                             const float2* __restrict__ x, const float* __restrict__ W,
                                                             float2* __restrict__ y, float4* __restrict__ part,
                                                             const KState* skip, int* err)
{
    if (skip && skip->done) return;   // uniform over the grid: the solve already finished
    // ring stage: the TR coupling rows, then x_b rows r0 - h .. r0 + TR + h.  Warps 0..7 consume
    // (two groups alternating the direct and transposed products), warp 8 produces the bulk
    // copies; a stage is refilled when the eight consumer warps have released it.
    extern __shared__ __align__(128) float wring[];
    __shared__ float4 xs[TR];                        // x_a rows of the tile: (x0.re, x0.im, x1.re, x1.im)
    __shared__ uint64_t full[NST], empty[NST];
    __shared__ int64_t spair[NST];                   // pair of each stage, written by the producer
    __shared__ int fail, issued;
    const int n1 = A.n1, ntile = gridDim.y;
    const int ch = blockIdx.x, tile = blockIdx.y, r0 = tile * TR;
    const int rows = min(TR, n1 - r0);
    const uint32_t bytes = (uint32_t)rows * ROWF * 4;
    const int own0 = A.own_start[ch], nown = A.own_start[ch + 1] - own0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lo = max(0, r0 - HO), hi = min(n1, r0 + TR + HO);
    const uint32_t xbytes = (uint32_t)(hi - lo) * 16;
    const int xoff = (lo - (r0 - HO)) * 4;   // floats
    if (tid == 0) {
        for (int q = 0; q < NST; q++) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 2 * NT / 32);
        }
        fail = 0;
        issued = 0;
        mbar_fence_init();
    }
    const float2* xa = x + (int64_t)ch * 2 * n1;
    if (tid < TR) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tid < rows) {
            float2 a = xa[2 * (r0 + tid)], b = xa[2 * (r0 + tid) + 1];
            v = make_float4(a.x, a.y, b.x, b.y);
        }
        xs[tid] = v;
    }
    // window rows outside the radial grid are never copied: zero them once in both stages (the
    // stored coupling is zero at those band positions, so the direct products need no range test)
    {
        const int wlo = lo - (r0 - HO), whi = hi - (r0 - HO);
        for (int i = tid; i < NST * NOUT; i += 2 * NT + 32) {
            int sg = i / NOUT, w = i - sg * NOUT;
            if (w < wlo || w >= whi)
                reinterpret_cast<float4*>(wring + sg * STAGE32 + TR * ROWF)[w] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    // consumer threads: group g = tid / NT, local index lt = tid % NT; for the k-th owned pair group
    // (k + g) % 2 forms the direct products of row r0 + lt, the other the transposed products of
    // output row r0 - h + lt, so every warp alternates the roles and both groups finish together
    const int grp = tid / NT, lt = tid % NT;
    const int r = r0 + lt;
    const bool direct_row = tid < 2 * NT && lt < TR && r < n1;
    __syncthreads();   // barriers initialised, xs staged, window margins zeroed
    float2 d0 = make_float2(0.f, 0.f), d1 = make_float2(0.f, 0.f);
    if (warp == 2 * NT / 32) {
        if (lane == 0) {
            for (int k = 0; k < nown; k++) {
                const int s = k % NST;
                if (k >= NST && !mbar_wait(&empty[s], (uint32_t)((k / NST - 1) & 1))) { fail = 1; break; }
                const int64_t p = A.own_pair[own0 + k];
                const int nb = A.own_nbr[own0 + k];
                float* st = wring + s * STAGE32;
                spair[s] = p;   // published by the arrive below
                // debug builds: copy from the buffers' starts instead of past their ends
                const int64_t pw = DG_INB(A, (p * n1 + r0 + rows) * ROWF <= A.nb_coup, 0) ? p : 0;
                const int nbw = DG_INB(A, ((int64_t)nb * n1 + hi) * 2 <= (int64_t)A.nch * n1 * 2, 1) ? nb : 0;
                fence_proxy_async();
                mbar_expect_tx(&full[s], bytes + xbytes);
                bulk_load(st, W + (pw * n1 + r0) * ROWF, bytes, &full[s]);
                bulk_load(st + TR * ROWF + xoff, x + ((int64_t)nbw * n1 + lo) * 2, xbytes, &full[s]);
                issued = k + 1;
            }
        }
    } else {
        // group 0's diagonal block (S + sign i tau H0) x_a, while the first copies are in flight
        if (grp == 0 && direct_row) {
            int ks = A.ch_kslot[ch];
            // bands with the rows innermost: diagonal d of row r is the float4 at (ks BDO + d) n1 + r
            const float4* Sk = reinterpret_cast<const float4*>(S) + (int64_t)ks * BDO * n1 + r;
            const float4* Hk = reinterpret_cast<const float4*>(H) + (int64_t)ks * BDO * n1 + r;
            const float* xaf = reinterpret_cast<const float*>(xa);
            float st = (float)(sign * A.tau);
#pragma unroll
            for (int d = 0; d < BDO; d++) {
                int rr = r + d - HO;
                if (rr < 0 || rr >= n1) continue;
                float4 xv = *reinterpret_cast<const float4*>(xaf + 4 * rr);
                float4 sv = Sk[(int64_t)d * n1];
                float4 hv = Hk[(int64_t)d * n1];
                float h00 = st * hv.x, h01 = st * hv.y, h10 = st * hv.z, h11 = st * hv.w;
                d0.x += sv.x * xv.x + sv.y * xv.z - (h00 * xv.y + h01 * xv.w);
                d0.y += sv.x * xv.y + sv.y * xv.w + (h00 * xv.x + h01 * xv.z);
                d1.x += sv.z * xv.x + sv.w * xv.z - (h10 * xv.y + h11 * xv.w);
                d1.y += sv.z * xv.y + sv.w * xv.w + (h10 * xv.x + h11 * xv.z);
            }
        }
        // the coupling sums are accumulated apart from the diagonal block and subtracted at the end
        float2 c0 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f);
        for (int k = 0; k < nown; k++) {
            const int s = k % NST;
            if (!mbar_wait(&full[s], (uint32_t)((k / NST) & 1))) { fail = 1; break; }
            const float* Ws = wring + s * STAGE32;
            const float4* Xs = reinterpret_cast<const float4*>(Ws + TR * ROWF);   // x_b row window
            if (((k + grp) & 1) == 0) {
                if (direct_row) {
#pragma unroll
                    for (int d = 0; d < BDO; d++) {
                        float4 xv = Xs[lt + d];   // row rr = r0 - h + (lt + d); zero outside the grid
                        float4 w = *reinterpret_cast<const float4*>(Ws + lt * ROWF + d * 4);
                        c0.x = fmaf(w.x, xv.x, c0.x); c0.x = fmaf(w.y, xv.z, c0.x);
                        c0.y = fmaf(w.x, xv.y, c0.y); c0.y = fmaf(w.y, xv.w, c0.y);
                        c1.x = fmaf(w.z, xv.x, c1.x); c1.x = fmaf(w.w, xv.z, c1.x);
                        c1.y = fmaf(w.z, xv.y, c1.y); c1.y = fmaf(w.w, xv.w, c1.y);
                    }
                }
            } else {
                // transposed: output row rb = r0 - h + j of channel b from the tile's rows of W_ab
                const int64_t p = spair[s];
                float4* pp = part + ((int64_t)p * ntile + tile) * NOUT;
                const int j = lt;
                float2 t0 = make_float2(0.f, 0.f), t1 = make_float2(0.f, 0.f);
                const int dlo = max(0, j - rows + 1), dhi = min(BDO - 1, j);
#pragma unroll 1
                for (int d = dlo; d <= dhi; d++) {
                    int lr = j - d;   // W row r0 + lr couples to column rb through diagonal d
                    float4 w = *reinterpret_cast<const float4*>(Ws + lr * ROWF + d * 4);
                    float4 xv = xs[lr];
                    // (W^T)[t][u] = W[u][t]
                    t0.x = fmaf(w.x, xv.x, t0.x); t0.x = fmaf(w.z, xv.z, t0.x);
                    t0.y = fmaf(w.x, xv.y, t0.y); t0.y = fmaf(w.z, xv.w, t0.y);
                    t1.x = fmaf(w.y, xv.x, t1.x); t1.x = fmaf(w.w, xv.z, t1.x);
                    t1.y = fmaf(w.y, xv.y, t1.y); t1.y = fmaf(w.w, xv.w, t1.y);
                }
                if (DG_INB(A, ((int64_t)p * ntile + tile) * NOUT + j < A.nb_part, 2))
                    pp[j] = make_float4(t0.x, t0.y, t1.x, t1.y);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);   // this warp is done with stage s
        }
        float sg = (float)sign;
        d0.x = fmaf(-sg, c0.x, d0.x); d0.y = fmaf(-sg, c0.y, d0.y);
        d1.x = fmaf(-sg, c1.x, d1.x); d1.y = fmaf(-sg, c1.y, d1.y);
    }
    __syncthreads();
    if (fail) {
        if (tid == 0) {
            atomicExch(err, 1);
            // copies still in flight target this block's shared memory: give the last ones issued
            // the same time limit before the block exits
            for (int k = max(0, issued - NST); k < issued; k++) mbar_wait(&full[k % NST], (uint32_t)((k / NST) & 1));
        }
        return;
    }
    // group 1's part of the rows to shared memory (the ring is free), group 0 adds it and stores
    float4* xch = reinterpret_cast<float4*>(wring);
    if (grp == 1 && direct_row) xch[lt] = make_float4(d0.x, d0.y, d1.x, d1.y);
    __syncthreads();
    if (grp == 0 && direct_row) {
        float4 o1 = xch[lt];
        int64_t o = (int64_t)ch * 2 * n1 + 2 * r;
        *reinterpret_cast<float4*>(y + o) = make_float4(d0.x + o1.x, d0.y + o1.y, d1.x + o1.z, d1.y + o1.w);
    }
}

__global__ void __launch_bounds__(NT) k_apply_gather32(OpView A, int sign, float2* __restrict__ y,
                                                       const float4* __restrict__ part,
                                                       const float2* __restrict__ bsub,
                                                       const float2* __restrict__ dv, double2* part_dot,
                                                       double* part_nrm, const KState* skip)
{
    if (skip && skip->done) return;
    const int n1 = A.n1, ntile = gridDim.y;
    const int ch = blockIdx.x, tile = blockIdx.y, r0 = tile * TR, tid = threadIdx.x;
    const int r = r0 + tid;
    const bool act = tid < TR && r < n1;
    float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
    if (act) {
        int64_t o = (int64_t)ch * 2 * n1 + 2 * r;
        float4 yv = *reinterpret_cast<const float4*>(y + o);
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int e = A.in_start[ch]; e < A.in_start[ch + 1]; e++) {
            const int64_t pb0 = (int64_t)A.in_pair[e] * ntile * NOUT;
            const float4* pp = part + pb0;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            const int64_t i0 = (int64_t)tile * NOUT + tid + HO;
            float4 v = DG_INB(A, pb0 + i0 < A.nb_part, 3) ? pp[i0] : z4;
            if (tid < HO && tile > 0) {
                const int64_t i1 = (int64_t)(tile - 1) * NOUT + TR + HO + tid;
                float4 u = DG_INB(A, pb0 + i1 < A.nb_part, 3) ? pp[i1] : z4;
                v.x += u.x; v.y += u.y; v.z += u.z; v.w += u.w;
            }
            if (tid >= TR - HO && tile + 1 < ntile) {   // tid < TR here
                const int64_t i2 = (int64_t)(tile + 1) * NOUT + tid - TR + HO;
                float4 u = DG_INB(A, pb0 + i2 < A.nb_part, 3) ? pp[i2] : z4;
                v.x += u.x; v.y += u.y; v.z += u.z; v.w += u.w;
            }
            t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
        }
        float sg = (float)sign;
        y0 = make_float2(fmaf(sg, t.x, yv.x), fmaf(sg, t.y, yv.y));
        y1 = make_float2(fmaf(sg, t.z, yv.z), fmaf(sg, t.w, yv.w));
        if (bsub) {
            float4 b = *reinterpret_cast<const float4*>(bsub + o);
            y0 = make_float2(b.x - y0.x, b.y - y0.y);
            y1 = make_float2(b.z - y1.x, b.w - y1.y);
        }
        *reinterpret_cast<float4*>(y + o) = make_float4(y0.x, y0.y, y1.x, y1.y);
    }
    if (part_dot || part_nrm) {
        double2 dsum = make_double2(0, 0);
        double nsum = 0;
        if (act) {
            int64_t o = (int64_t)ch * 2 * n1 + 2 * r;
            if (dv) {
                float4 a = *reinterpret_cast<const float4*>(dv + o);
                dsum.x = (double)a.x * y0.x + (double)a.y * y0.y + (double)a.z * y1.x + (double)a.w * y1.y;
                dsum.y = (double)a.x * y0.y - (double)a.y * y0.x + (double)a.z * y1.y - (double)a.w * y1.x;
            }
            nsum = (double)y0.x * y0.x + (double)y0.y * y0.y + (double)y1.x * y1.x + (double)y1.y * y1.y;
        }
        block_reduce_store(dsum, nsum, part_dot, part_nrm, (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
    }
}

// ---------------------------------------------------------------------------------------------
// Refinement residual r = A_- psi - A_+ x = S (psi - x) - i tau H0 (psi + x) + (W - W^T)(psi + x)
// in double-float, from u = psi + x and v = psi - x split into (re hi, re lo, im hi, im lo) and stored
// type-major ([channel][DKB type][slot], so a type's rows are contiguous 16 B records), and,
// when *need_b is set (the first pass of a step), b = A_- psi in FP32 products for the tolerance
// scale ||b||.  Owner pass: the direct coupling sums W_ab u_b of channel a to r_out (W_ab psi_b to
// b_out); partials of the transposed products to part_r (the unnormalised double-float accumulators
// (s, c) of the four components, two float4 per row: no FP64 instruction in this pass) and part_b.
// Gather pass: the diagonal block S v - i tau H0 u of the channel (latency-bound band reads at high
// occupancy, so the owner pass's warps spend their time on the coupling), plus the direct sums,
// minus the partials.
// ---------------------------------------------------------------------------------------------
namespace {
constexpr int NSTD = 2;          // ring depth of the double-float pass
// floats per stage: hi and lo words of the TR coupling rows, the u_b row window (type 0, type 1) and,
// on a step's first pass, the FP32 psi_b row window (both types per 16-byte row)
constexpr int STAGE_DF = 2 * TR * ROWF + NOUT * 8 + NOUT * 4;
constexpr int PS_OFF = 2 * TR * ROWF + NOUT * 8;      // psi_b window offset in a stage (floats)
// offset bytes of one (pair, tile): direct rows r0 + [0, TR) at [0, TR), transposed output rows
// r0 - h + [0, NOUT) at [NOUT, 2 NOUT); the stage keeps them after its floats
constexpr int SIG_BYTES = 2 * NOUT;
// u-window sums: row r of channel ch at ch * us_stride(n1) + US_PAD + r; US_PAD zero rows on both
// sides (the offset kernel reads four consecutive rows from r0 - h on) and a stride that keeps the
// four-row groups of the offset kernel 8- or 16-byte aligned
constexpr int US_PAD = 8;
__host__ __device__ constexpr int us_stride(int n1) { return ((n1 + 2 * US_PAD) + 3) & ~3; }
constexpr int STAGE_DFS = STAGE_DF + SIG_BYTES / 4;   // floats per stage with the offset bytes
}

// Window sums of the split vector u = psi + x for the offsets of the owner pass:
// US[ch][r] = sum over rows rr in [r - h, r + h] of max(|re hi|, |im hi|) over both DKB types of
// u_ch(rr).  Every product of a row's direct sum (or of a transposed output row's sum) takes one u
// factor from that window, so US bounds the u side of the sum of |products|.
__global__ void __launch_bounds__(128) k_usum(OpView A, const float4* __restrict__ u, float* __restrict__ US)
{
    __shared__ float m[128 + 2 * HO];
    const int n1 = A.n1, ch = blockIdx.y, r0 = blockIdx.x * 128;
    const float4* u0 = u + (int64_t)ch * 2 * n1;   // type-major: type 0 rows, then type 1 rows
    const float4* u1 = u0 + n1;
    for (int i = threadIdx.x; i < 128 + 2 * HO; i += 128) {
        const int rr = r0 - HO + i;
        float v = 0.f;
        if (rr >= 0 && rr < n1) {
            const float4 a = u0[rr], b = u1[rr];
            v = fmaxf(fmaxf(fabsf(a.x), fabsf(a.z)), fmaxf(fabsf(b.x), fabsf(b.z)));
        }
        m[i] = v;
    }
    __syncthreads();
    const int r = r0 + threadIdx.x;
    if (r < n1) {
        float sum = 0.f;
        for (int d = 0; d < BDO; d++) sum += m[threadIdx.x + d];
        US[(int64_t)ch * us_stride(n1) + US_PAD + r] = sum;
    }
}

// Offsets of the owner pass's accumulators (df_fma_off): for every pair p and radial tile, one
// byte per direct row r (the sum of W_p(r, .) u_b over the row's band) and per transposed output
// row R (the sum of W_p(., .)^T u_a reaching R).  The bound of the sum of |products|:
//  - W_p = sum over its multipoles l of cA_l K_l + cB_l KT_l (the grouped assembly's coefficients)
//    with K_l = sum_n m_n G^n_l and G^n_l = sum_c s_lc(t) M_lcn (the static pulse matrices); so
//    every entry of row r of W_p is at most Mb(r) = sum_l S_l (|cA_l| eA_l(r) + |cB_l| eB_l(r)),
//    S_l = sum_c |s_lc(t)|, eA_l = sum_n |m_n| E_ln, eB_l = sum_n |m'_n| E_ln (m = (1, ka, kb, ka kb),
//    m' = (1, kb, ka, ka kb): one pair group shares them) and E_ln(r) the largest |M_lcn| entry of
//    row r and of column r over c (KT reads G at the transposed position, i.e. along column r);
//  - a direct row takes two entries of each of its band positions, against u_b in [r - h, r + h]:
//    B = 2 Mb(r) US_b(r); a transposed output row R takes two entries of rows R - h .. R + h against
//    u_a on those rows: B = 2 max_{|lr - R| <= h} Mb(lr) US_a(R), the max taken from Ew, the
//    13-row window maxima of E.
// All factors are rounded up or carry the 1.0625 of df_offset_byte.  Grid: (tiles, chunks of the
// grouped assembly); a block forms its rows' eA, eB once and then spends a few FMAs per pair.
// the pairs of one chunk for one thread's four row slots (NL = the chunk's multipoles): the chunk's
// kappa-weighted envelopes eA, eB at the four rows, then per pair the bound of each slot and its
// offset byte, the four packed into one store
template <int NL>
__device__ __forceinline__ void sigma_pairs(const AsmChunk& ch, const int* __restrict__ lsel,
                                            const float* __restrict__ Et, int n1, int usn, const int (&row)[4],
                                            const bool (&valid)[4], bool direct, int slot0, int tile, int ntile,
                                            const int* sp, const int* sa, const int* sb, const float2* scf,
                                            const float* __restrict__ US, unsigned char* __restrict__ sig)
{
    const float fa = fabsf((float)ch.ka), fb = fabsf((float)ch.kb);
    const float mk[4] = {1.f, fa, fb, fa * fb}, mt[4] = {1.f, fb, fa, fa * fb};
    float eA[4][NL], eB[4][NL];   // [slot][multipole]
#pragma unroll
    for (int j = 0; j < NL; j++) {
        const float* El = Et + (int64_t)lsel[j] * 4 * n1;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            eA[i][j] = 0.f;
            eB[i][j] = 0.f;
            if (valid[i]) {
#pragma unroll
                for (int n = 0; n < 4; n++) {
                    const float v = El[(int64_t)n * n1 + row[i]];
                    eA[i][j] = fmaf(mk[n], v, eA[i][j]);
                    eB[i][j] = fmaf(mt[n], v, eB[i][j]);
                }
            }
        }
    }
    // the four rows' u-window sums are one aligned group (zero margins outside the grid): one
    // 16-byte load for the direct slots (rows r0 + 4 t), two 8-byte ones for the transposed slots
    // (rows r0 - h + 4 t, two rows off the 16-byte grid)
    // a group with a valid slot has rows within [-h, n1 + 2], inside the margins; the unused slots
    // TR .. NOUT - 1 and groups past the grid load nothing
    const bool any = valid[0] || valid[1] || valid[2] || valid[3];
    const int64_t uo = US_PAD + row[0];
    for (int q = 0; q < ch.count; q++) {
        const float* ub = US + (int64_t)(direct ? sb[q] : sa[q]) * usn + uo;
        float uw[4] = {0.f, 0.f, 0.f, 0.f};
        if (!any) {
        } else if (direct) {
            const float4 t = *reinterpret_cast<const float4*>(ub);
            uw[0] = t.x; uw[1] = t.y; uw[2] = t.z; uw[3] = t.w;
        } else {
            const float2 t0 = *reinterpret_cast<const float2*>(ub), t1 = *reinterpret_cast<const float2*>(ub + 2);
            uw[0] = t0.x; uw[1] = t0.y; uw[2] = t1.x; uw[3] = t1.y;
        }
        float2 w[NL];   // zero for multipoles the pair lacks
#pragma unroll
        for (int j = 0; j < NL; j++) w[j] = scf[q * ASM_MAX_NL + j];
        unsigned int packed = 0;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            float Mb = 0.f;
#pragma unroll
            for (int j = 0; j < NL; j++) Mb = fmaf(w[j].x, eA[i][j], fmaf(w[j].y, eB[i][j], Mb));
            packed |= df_offset_byte(valid[i] ? 2.f * Mb * uw[i] : 0.f) << (8 * i);
        }
        *reinterpret_cast<unsigned int*>(sig + ((int64_t)sp[q] * ntile + tile) * SIG_BYTES + slot0) = packed;
    }
}

__global__ void __launch_bounds__(SIG_BYTES / 4) k_own_sigma(OpView A, const AsmChunk* __restrict__ chunks,
                                                              int nchunks, const int* __restrict__ gpair,
                                                              const float4* __restrict__ gcoef,
                                                              const double* __restrict__ s, const float* __restrict__ E,
                                                              const float* __restrict__ Ew,
                                                              const float* __restrict__ US,
                                                              unsigned char* __restrict__ sig)
{
    __shared__ int sp[ASM_CHUNK], sa[ASM_CHUNK], sb[ASM_CHUNK];
    __shared__ float2 scf[ASM_CHUNK * ASM_MAX_NL];   // (|cA_l| S_l, |cB_l| S_l)
    const int n1 = A.n1, tile = blockIdx.x, ntile = gridDim.x;
    // each thread owns four consecutive slots of the record: slot0 .. slot0 + 3 (a group never
    // straddles the direct / transposed boundary: TR and NOUT are multiples of 4)
    static_assert(TR % 4 == 0 && NOUT % 4 == 0, "slot groups of four");
    const int slot0 = 4 * threadIdx.x;
    const bool direct = slot0 < TR;
    int row[4];
    bool valid[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int sl = slot0 + i;
        row[i] = direct ? tile * TR + sl : tile * TR - HO + (sl - NOUT);
        valid[i] = (direct || sl >= NOUT) && row[i] >= 0 && row[i] < n1;
    }
    const float* Et = direct ? E : Ew;
    const int usn = us_stride(n1);
    for (int c = blockIdx.y; c < nchunks; c += gridDim.y) {
        const AsmChunk ch = chunks[c];
        __syncthreads();   // the previous chunk's staged values are no longer read
        for (int i = threadIdx.x; i < ch.count; i += blockDim.x) {
            const int p = gpair[ch.first + i];
            sp[i] = p;
            sa[i] = A.pair_a[p];
            sb[i] = A.pair_b[p];
        }
        for (int i = threadIdx.x; i < ch.count * ASM_MAX_NL; i += blockDim.x) {
            const int l = chunks[c].l[i % ASM_MAX_NL];   // from memory: no local copy of the record
            const float S = (float)((fabs(s[3 * l]) + fabs(s[3 * l + 1]) + fabs(s[3 * l + 2])) * (1.0 + 1e-6));
            const float4 cf = gcoef[(int64_t)ch.first * ASM_MAX_NL + i];   // (cA hi, lo, cB hi, lo)
            scf[i] = make_float2(fabsf(cf.x) * S, fabsf(cf.z) * S);
        }
        __syncthreads();
        switch (ch.nl) {
        case 1: sigma_pairs<1>(ch, chunks[c].l, Et, n1, usn, row, valid, direct, slot0, tile, ntile, sp, sa, sb, scf,
                               US, sig); break;
        case 2: sigma_pairs<2>(ch, chunks[c].l, Et, n1, usn, row, valid, direct, slot0, tile, ntile, sp, sa, sb, scf,
                               US, sig); break;
        case 3: sigma_pairs<3>(ch, chunks[c].l, Et, n1, usn, row, valid, direct, slot0, tile, ntile, sp, sa, sb, scf,
                               US, sig); break;
        default: sigma_pairs<4>(ch, chunks[c].l, Et, n1, usn, row, valid, direct, slot0, tile, ntile, sp, sa, sb, scf,
                                US, sig); break;
        }
    }
}

// Warp roles: two groups of four consumer warps alternate the direct products (row r0 + lt) and the
// transposed products (output row r0 - h + lt) from pair to pair; warp 8 is the producer that keeps
// the NSTD-deep ring of bulk copies filled.  A stage is refilled when all eight consumer warps have
// released it (an "empty" mbarrier), so the groups drift freely within the ring instead of meeting
// at a block barrier for every pair.
constexpr int NTHR_OWN = 2 * NT + 32;

// one double-float multiply-add: fixed-binade form (df_fma_off) or the Dot2 form (df_fma)
template <bool OFF>
__device__ __forceinline__ void acc_fma(DfAcc& a, float wh, float wl, float xh, float xl)
{
    if constexpr (OFF) df_fma_off(a, wh, wl, xh, xl);
    else df_fma(a, wh, wl, xh, xl);
}

// direct products of one owned pair for row r0 + lt: acc += W(r, .) u_b over the band (and, NB, the
// FP32 products of b = A_- psi), from the stage's coupling rows and row windows
template <bool OFF, bool NB>
__device__ __forceinline__ void own_direct(DfAcc (&acc)[4], float (&db)[4], const float* Hs, const float* Ls,
                                           const float4* Us0, const float4* Us1, const float4* Ps, int lt)
{
#pragma unroll
    for (int d = 0; d < BDO; d++) {
        // window index of row rr = r + d - h: rr - (r0 - h) = lt + d; rows outside the grid are zero
        // in the window and in W
        const float4 x0 = Us0[lt + d], x1 = Us1[lt + d];
        const float4 wh = *reinterpret_cast<const float4*>(Hs + lt * ROWF + d * 4);
        const float4 wl = *reinterpret_cast<const float4*>(Ls + lt * ROWF + d * 4);
        // W[t][u] = (w.x, w.y ; w.z, w.w)
        acc_fma<OFF>(acc[0], wh.x, wl.x, x0.x, x0.y); acc_fma<OFF>(acc[0], wh.y, wl.y, x1.x, x1.y);
        acc_fma<OFF>(acc[1], wh.x, wl.x, x0.z, x0.w); acc_fma<OFF>(acc[1], wh.y, wl.y, x1.z, x1.w);
        acc_fma<OFF>(acc[2], wh.z, wl.z, x0.x, x0.y); acc_fma<OFF>(acc[2], wh.w, wl.w, x1.x, x1.y);
        acc_fma<OFF>(acc[3], wh.z, wl.z, x0.z, x0.w); acc_fma<OFF>(acc[3], wh.w, wl.w, x1.z, x1.w);
        if (NB) {   // psi_b window rows outside the grid are zero, as u_b's
            const float4 q = Ps[lt + d];
            db[0] += wh.x * q.x + wh.y * q.z;
            db[1] += wh.x * q.y + wh.y * q.w;
            db[2] += wh.z * q.x + wh.w * q.z;
            db[3] += wh.z * q.y + wh.w * q.w;
        }
    }
}

// NEED_B: the pass also forms the FP32 products of b = A_- psi (a step's first pass).  The flag is
// read on the device (a captured graph replays one launch for every pass), so both instantiations
// are launched and the one that does not match the flag returns at once.  OFF: the accumulators
// take the fixed-binade form with the offsets of k_own_sigma (six FP32 operations per multiply-add,
// error of order 2^-48 times the offset), else the Dot2 form (ten operations, error of order 2^-48
// times the running sum); the host picks OFF from the solve's tolerance.
template <bool NEED_B, bool OFF>
__global__ void __launch_bounds__(NTHR_OWN) k_residual_own_df(OpView A, const float4* __restrict__ u,
                                                             const float2* __restrict__ psi32,
                                                             const float* __restrict__ Wh, const float* __restrict__ Wl,
                                                             double2* __restrict__ r_out, float2* __restrict__ b_out,
                                                             float4* __restrict__ part_r, float4* __restrict__ part_b,
                                                             const unsigned char* __restrict__ sig,
                                                             const int* need_b_flag, int* err)
{
    if ((*need_b_flag != 0) != NEED_B) return;   // uniform over the grid
    constexpr bool need_b = NEED_B;
    // ring stage: hi words, lo words of the TR coupling rows, then u_b rows r0 - h .. r0 + TR + h
    extern __shared__ __align__(128) float wring[];
    __shared__ float4 us0[TR], us1[TR];              // u_a rows of DKB type 0 and 1 (split complex)
    __shared__ float4 ps[TR];                        // psi_a rows in FP32: (p0.re, p0.im, p1.re, p1.im)
    __shared__ uint64_t full[NSTD], empty[NSTD];
    __shared__ int64_t spair[NSTD];                  // pair of each stage
    __shared__ int fail, issued;
    const int n1 = A.n1, ntile = gridDim.y;
    const int ch = blockIdx.x, tile = blockIdx.y, r0 = tile * TR;
    const int rows = min(TR, n1 - r0);
    const uint32_t bytes = (uint32_t)rows * ROWF * 4;
    const int own0 = A.own_start[ch], nown = A.own_start[ch + 1] - own0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int stage_f = STAGE_DFS;
    // u_b window: rows [lo, hi) land at window index lo - (r0 - h)
    const int lo = max(0, r0 - HO), hi = min(n1, r0 + TR + HO);
    // u is type-major ([channel][type][slot]): a type's window is one contiguous copy of 16 B rows
    const uint32_t ubytes = (uint32_t)(hi - lo) * 16;
    const int uoff = (lo - (r0 - HO)) * 4;   // floats
    if (tid == 0) {
        for (int q = 0; q < NSTD; q++) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 2 * NT / 32);
        }
        fail = 0;
        issued = 0;
        mbar_fence_init();
    }
    const float4* ua0 = u + (int64_t)ch * 2 * n1;   // type 0 rows of channel ch, then type 1
    const float4* ua1 = ua0 + n1;
    const float2* pa = psi32 + (int64_t)ch * 2 * n1;
    if (tid < TR) {
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        bool in = tid < rows;
        us0[tid] = in ? ua0[r0 + tid] : z;
        us1[tid] = in ? ua1[r0 + tid] : z;
        if (need_b) ps[tid] = in ? *reinterpret_cast<const float4*>(pa + 2 * (r0 + tid)) : z;
    }
    // window rows outside the radial grid are never copied: zero them once in both stages, so the
    // direct products need no range test (the stored coupling is zero at those band positions)
    {
        const int wlo = lo - (r0 - HO), whi = hi - (r0 - HO);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = tid; i < NSTD * NOUT; i += NTHR_OWN) {
            int sg = i / NOUT, w = i - sg * NOUT;
            if (w < wlo || w >= whi) {
                float4* Uz = reinterpret_cast<float4*>(wring + sg * stage_f + 2 * TR * ROWF);   // [type][window]
                Uz[w] = z;
                Uz[NOUT + w] = z;
                Uz[2 * NOUT + w] = z;   // psi_b window
            }
        }
    }
    // consumer threads: group g = tid / NT (0 or 1), local index lt = tid % NT.  For the k-th owned
    // pair, group (k + g) % 2 forms the direct products of row r0 + lt and the other group the
    // transposed products of output row r0 - h + lt: every warp alternates the two roles, so both
    // groups finish together whatever the relative cost of the roles.
    const int grp = tid / NT, lt = tid % NT;
    const int r = r0 + lt;
    const bool direct_row = tid < 2 * NT && lt < TR && r < n1;
    __syncthreads();   // barriers initialised, us and ps staged
    DfAcc dd[4];
    for (int k = 0; k < 4; k++) df_zero(dd[k]);
    float db[4] = {0.f, 0.f, 0.f, 0.f};
    if (warp == 2 * NT / 32) {
        // producer
        if (lane == 0) {
            for (int k = 0; k < nown; k++) {
                const int s = k % NSTD;
                if (k >= NSTD && !mbar_wait(&empty[s], (uint32_t)((k / NSTD - 1) & 1))) { fail = 1; break; }
                const int64_t p = A.own_pair[own0 + k];
                const int nb = A.own_nbr[own0 + k];
                float* st = wring + s * stage_f;
                spair[s] = p;   // published by the arrive below
                // debug builds: copy from the buffers' starts instead of past their ends
                const int64_t pw = DG_INB(A, (p * n1 + r0 + rows) * ROWF <= A.nb_coup, 0) ? p : 0;
                const int nbw = DG_INB(A, ((int64_t)nb * 2 + 1) * n1 + hi <= (int64_t)A.nch * n1 * 2, 1) ? nb : 0;
                fence_proxy_async();
                mbar_expect_tx(&full[s], 2 * bytes + (need_b ? 3 : 2) * ubytes + (OFF ? SIG_BYTES : 0));
                bulk_load(st, Wh + (pw * n1 + r0) * ROWF, bytes, &full[s]);
                bulk_load(st + TR * ROWF, Wl + (pw * n1 + r0) * ROWF, bytes, &full[s]);
                bulk_load(st + 2 * TR * ROWF + uoff, u + ((int64_t)nbw * 2) * n1 + lo, ubytes, &full[s]);
                bulk_load(st + 2 * TR * ROWF + NOUT * 4 + uoff, u + ((int64_t)nbw * 2 + 1) * n1 + lo, ubytes, &full[s]);
                if (need_b)   // psi_b rows [lo, hi): 16 B each (both types), the state's own order
                    bulk_load(st + PS_OFF + uoff, psi32 + ((int64_t)nbw * n1 + lo) * 2, ubytes, &full[s]);
                if (OFF)   // this pair-tile's accumulator offsets
                    bulk_load(st + STAGE_DF, sig + ((int64_t)pw * ntile + tile) * SIG_BYTES, SIG_BYTES, &full[s]);
                issued = k + 1;
            }
        }
    } else {
        for (int k = 0; k < nown; k++) {
            const int s = k % NSTD;
            if (!mbar_wait(&full[s], (uint32_t)((k / NSTD) & 1))) { fail = 1; break; }
            const float* Hs = wring + s * stage_f;
            const float* Ls = Hs + TR * ROWF;
            const float4* Us0 = reinterpret_cast<const float4*>(Hs + 2 * TR * ROWF);   // [row window], type 0
            const float4* Us1 = Us0 + NOUT;                                             // type 1
            const unsigned char* Sg = reinterpret_cast<const unsigned char*>(Hs + STAGE_DF);   // offsets
            if (((k + grp) & 1) == 0) {
                if (direct_row) {
                    const float4* Ps = reinterpret_cast<const float4*>(Hs + PS_OFF);   // psi_b window
                    if constexpr (OFF) {
                        // this pair's sums in fixed-binade accumulators (df_fma_off), then added to dd
                        const float sg = df_offset(Sg[lt]);
                        DfAcc aa[4];
                        for (int q = 0; q < 4; q++) { aa[q].s = sg; aa[q].c = 0.f; }
                        own_direct<true, NEED_B>(aa, db, Hs, Ls, Us0, Us1, Ps, lt);
                        for (int q = 0; q < 4; q++) {
                            // the bound held: the sum stayed within 2^(k-2) = sg / 6 of the offset
                            (void)DG_INB(A, fabsf(aa[q].s - sg) <= 0.1667f * sg, 6);
                            DfAcc v = {aa[q].s - sg, aa[q].c};
                            df_add(dd[q], v, 1.f);
                        }
                    } else {
                        own_direct<false, NEED_B>(dd, db, Hs, Ls, Us0, Us1, Ps, lt);
                    }
                }
            } else {
                const int64_t p = spair[s];
                float4* pr = part_r + (((int64_t)p * ntile + tile) * NOUT) * 2;
                float4* pbp = part_b + ((int64_t)p * ntile + tile) * NOUT;
                const int j = lt;   // one output row per thread (NOUT == NT)
                const bool slot_ok = DG_INB(A, ((int64_t)p * ntile + tile) * NOUT + j < A.nb_part, 2);
                DfAcc tt[4];
                const float sg = OFF ? df_offset(Sg[NOUT + j]) : 0.f;   // Dot2 form: from zero
                for (int q = 0; q < 4; q++) { tt[q].s = sg; tt[q].c = 0.f; }
                float tb[4] = {0.f, 0.f, 0.f, 0.f};
                // diagonals whose W row r0 + j - d lies in the tile (a rolled loop: with the direct
                // products unrolled, unrolling this one too overflows the instruction cache)
                const int dlo = max(0, j - rows + 1), dhi = min(BDO - 1, j);
#pragma unroll 1
                for (int d = dlo; d <= dhi; d++) {
                    const int lr = j - d;
                    float4 wh = *reinterpret_cast<const float4*>(Hs + lr * ROWF + d * 4);
                    float4 wl = *reinterpret_cast<const float4*>(Ls + lr * ROWF + d * 4);
                    float4 x0 = us0[lr], x1 = us1[lr];
                    // (W^T)[t][u] = W[u][t]
                    acc_fma<OFF>(tt[0], wh.x, wl.x, x0.x, x0.y); acc_fma<OFF>(tt[0], wh.z, wl.z, x1.x, x1.y);
                    acc_fma<OFF>(tt[1], wh.x, wl.x, x0.z, x0.w); acc_fma<OFF>(tt[1], wh.z, wl.z, x1.z, x1.w);
                    acc_fma<OFF>(tt[2], wh.y, wl.y, x0.x, x0.y); acc_fma<OFF>(tt[2], wh.w, wl.w, x1.x, x1.y);
                    acc_fma<OFF>(tt[3], wh.y, wl.y, x0.z, x0.w); acc_fma<OFF>(tt[3], wh.w, wl.w, x1.z, x1.w);
                    if (need_b) {
                        float4 q = ps[lr];
                        tb[0] += wh.x * q.x + wh.z * q.z;
                        tb[1] += wh.x * q.y + wh.z * q.w;
                        tb[2] += wh.y * q.x + wh.w * q.z;
                        tb[3] += wh.y * q.y + wh.w * q.w;
                    }
                }
                if (slot_ok) {
                    if (OFF)
                        for (int q = 0; q < 4; q++) (void)DG_INB(A, fabsf(tt[q].s - sg) <= 0.1667f * sg, 6);
                    // (s - offset, c): exact (the Dot2 form has offset 0), the unnormalised pair the
                    // gather pass adds
                    pr[2 * j] = make_float4(tt[0].s - sg, tt[0].c, tt[1].s - sg, tt[1].c);
                    pr[2 * j + 1] = make_float4(tt[2].s - sg, tt[2].c, tt[3].s - sg, tt[3].c);
                    if (need_b) pbp[j] = make_float4(tb[0], tb[1], tb[2], tb[3]);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);   // this warp is done with stage s
        }
    }
    __syncthreads();
    if (fail) {
        if (tid == 0) {
            atomicExch(err, 1);
            // copies still in flight target this block's shared memory: give the last ones issued
            // the same time limit before the block exits
            for (int k = max(0, issued - NSTD); k < issued; k++) mbar_wait(&full[k % NSTD], (uint32_t)((k / NSTD) & 1));
        }
        return;
    }
    // group 1's direct sums to shared memory (the ring is free: every copy has been consumed),
    // group 0 adds them in a fixed order and stores the row
    float4* xch = reinterpret_cast<float4*>(wring);   // [NT][3]: (s, c) x 4, then the FP32 b sums
    if (grp == 1 && direct_row) {
        xch[3 * lt] = make_float4(dd[0].s, dd[0].c, dd[1].s, dd[1].c);
        xch[3 * lt + 1] = make_float4(dd[2].s, dd[2].c, dd[3].s, dd[3].c);
        xch[3 * lt + 2] = make_float4(db[0], db[1], db[2], db[3]);
    }
    __syncthreads();
    if (grp == 0 && direct_row) {
        float4 a0 = xch[3 * lt], a1 = xch[3 * lt + 1], a2 = xch[3 * lt + 2];
        DfAcc o0 = {a0.x, a0.y}, o1 = {a0.z, a0.w}, o2 = {a1.x, a1.y}, o3 = {a1.z, a1.w};
        df_add(dd[0], o0, 1.f);
        df_add(dd[1], o1, 1.f);
        df_add(dd[2], o2, 1.f);
        df_add(dd[3], o3, 1.f);
        int64_t o = (int64_t)ch * 2 * n1 + 2 * r;
        r_out[o] = make_double2(df_value(dd[0]), df_value(dd[1]));
        r_out[o + 1] = make_double2(df_value(dd[2]), df_value(dd[3]));
        if (need_b)
            *reinterpret_cast<float4*>(b_out + o) =
                make_float4(db[0] + a2.x, db[1] + a2.y, db[2] + a2.z, db[3] + a2.w);
    }
}

// r_b -= sum of the transposed partials (own tile and the neighbours' halo rows, fixed order) in
// double-float; partials of ||r||^2 and, on a step's first pass, of ||b||^2
__global__ void __launch_bounds__(NT) k_residual_gather_df(OpView A, const float2* __restrict__ S,
                                                           const float2* __restrict__ Ht,
                                                           const float4* __restrict__ u,
                                                           const float4* __restrict__ v,
                                                           const float2* __restrict__ psi32,
                                                           double2* __restrict__ r_out,
                                                           const float2* __restrict__ b_out,
                                                           const float4* __restrict__ part_r,
                                                           const float4* __restrict__ part_b,
                                                           const int* need_b_flag, double* pn_r, double* pn_b)
{
    const bool need_b = *need_b_flag != 0;
    const int n1 = A.n1, ntile = gridDim.y;
    const int ch = blockIdx.x, tile = blockIdx.y, r0 = tile * TR, tid = threadIdx.x;
    const int r = r0 + tid;
    double nr = 0, nb = 0;
    if (tid < TR && r < n1) {
        int64_t o = (int64_t)ch * 2 * n1 + 2 * r;
        // diagonal block: S (psi - x) - i tau H0 (psi + x), and b's FP32 part (S - i tau H0) psi
        const float4* ua = u + (int64_t)ch * 2 * n1;   // type-major: type 0 rows, then type 1 rows
        const float4* va = v + (int64_t)ch * 2 * n1;
        const float2* pa = psi32 + (int64_t)ch * 2 * n1;
        int ks = A.ch_kslot[ch];
        // bands with the rows innermost: diagonal d of row r is the 32-byte record (ks BDO + d) n1 + r
        const float4* Sk = reinterpret_cast<const float4*>(S) + ((int64_t)ks * BDO * n1 + r) * 2;
        const float4* Hk = reinterpret_cast<const float4*>(Ht) + ((int64_t)ks * BDO * n1 + r) * 2;
        DfAcc acc[4];   // (type 0 re, im, type 1 re, im)
        for (int k = 0; k < 4; k++) df_zero(acc[k]);
        float bb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int d = 0; d < BDO; d++) {
            int rr = r + d - HO;
            if (rr < 0 || rr >= n1) continue;
            float4 u0 = ua[rr], u1 = ua[n1 + rr], v0 = va[rr], v1 = va[n1 + rr];
            float4 pv = need_b ? *reinterpret_cast<const float4*>(pa + 2 * rr) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 sq[2] = {Sk[(int64_t)d * n1 * 2], Sk[(int64_t)d * n1 * 2 + 1]};   // entries (0 1 | 2 3)
            const float4 hq[2] = {Hk[(int64_t)d * n1 * 2], Hk[(int64_t)d * n1 * 2 + 1]};
            for (int t = 0; t < 2; t++) {
                const float2 s0 = make_float2(sq[t].x, sq[t].y), s1 = make_float2(sq[t].z, sq[t].w);
                const float2 h0 = make_float2(hq[t].x, hq[t].y), h1 = make_float2(hq[t].z, hq[t].w);
                // re: S v_re + tau H u_im ;  im: S v_im - tau H u_re
                df_fma(acc[2 * t], s0.x, s0.y, v0.x, v0.y);
                df_fma(acc[2 * t], s1.x, s1.y, v1.x, v1.y);
                df_fma(acc[2 * t], h0.x, h0.y, u0.z, u0.w);
                df_fma(acc[2 * t], h1.x, h1.y, u1.z, u1.w);
                df_fma(acc[2 * t + 1], s0.x, s0.y, v0.z, v0.w);
                df_fma(acc[2 * t + 1], s1.x, s1.y, v1.z, v1.w);
                df_fma(acc[2 * t + 1], -h0.x, -h0.y, u0.x, u0.y);
                df_fma(acc[2 * t + 1], -h1.x, -h1.y, u1.x, u1.y);
                bb[2 * t] += s0.x * pv.x + s1.x * pv.z + h0.x * pv.y + h1.x * pv.w;
                bb[2 * t + 1] += s0.x * pv.y + s1.x * pv.w - h0.x * pv.x - h1.x * pv.z;
            }
        }
        // + the owner pass's direct coupling sums W (psi + x)
        double2 y0 = r_out[o], y1 = r_out[o + 1];
        const double yv[4] = {y0.x, y0.y, y1.x, y1.y};
        for (int k = 0; k < 4; k++) {
            float2 h = df_split_bits(yv[k]);
            DfAcc t = {h.x, h.y};
            df_add(acc[k], t, 1.f);
        }
        float4 bv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (need_b) {
            float4 bo = *reinterpret_cast<const float4*>(b_out + o);
            bv = make_float4(bb[0] + bo.x, bb[1] + bo.y, bb[2] + bo.z, bb[3] + bo.w);
        }
        for (int e = A.in_start[ch]; e < A.in_start[ch + 1]; e++) {
            int64_t p = A.in_pair[e];
            const float4* pr = part_r + (int64_t)p * ntile * NOUT * 2;
            const float4* pb = part_b + (int64_t)p * ntile * NOUT;
            int js[3], ts[3], nj = 0;
            js[nj] = tid + HO; ts[nj++] = tile;
            if (tid < HO && tile > 0) { js[nj] = TR + HO + tid; ts[nj++] = tile - 1; }
            if (tid >= TR - HO && tile + 1 < ntile) { js[nj] = tid - TR + HO; ts[nj++] = tile + 1; }
            for (int q = 0; q < nj; q++) {
                int64_t i = (int64_t)ts[q] * NOUT + js[q];
                if (!DG_INB(A, p * ntile * NOUT + i < A.nb_part, 3)) continue;
                float4 a = pr[2 * i], c = pr[2 * i + 1];
                DfAcc t0 = {a.x, a.y}, t1 = {a.z, a.w}, t2 = {c.x, c.y}, t3 = {c.z, c.w};
                df_add(acc[0], t0, -1.f);
                df_add(acc[1], t1, -1.f);
                df_add(acc[2], t2, -1.f);
                df_add(acc[3], t3, -1.f);
                if (need_b) {
                    float4 w = pb[i];
                    bv.x -= w.x; bv.y -= w.y; bv.z -= w.z; bv.w -= w.w;
                }
            }
        }
        y0 = make_double2(df_value(acc[0]), df_value(acc[1]));
        y1 = make_double2(df_value(acc[2]), df_value(acc[3]));
        r_out[o] = y0;
        r_out[o + 1] = y1;
        nr = y0.x * y0.x + y0.y * y0.y + y1.x * y1.x + y1.y * y1.y;
        nb = (double)bv.x * bv.x + (double)bv.y * bv.y + (double)bv.z * bv.z + (double)bv.w * bv.w;
    }
    int64_t slot = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    block_reduce_store(make_double2(0, 0), nr, nullptr, pn_r, slot);
    if (need_b) block_reduce_store(make_double2(0, 0), nb, nullptr, pn_b, slot);
}

size_t residual_own_df_smem() { return (size_t)NSTD * STAGE_DFS * sizeof(float); }

void launch_residual_offsets(cudaStream_t st, const OpView& A, const AsmChunk* chunks, int nchunks, const int* gpair,
                             const float4* gcoef, const double* s, const float* E, const float* Ew, float* US,
                             unsigned char* sig, const float4* u)
{
    const int ntile = (A.n1 + TR - 1) / TR;
    k_usum<<<dim3((A.n1 + 127) / 128, A.nch), 128, 0, st>>>(A, u, US);
    k_own_sigma<<<dim3(ntile, (unsigned)(nchunks < 65535 ? nchunks : 65535)), SIG_BYTES / 4, 0, st>>>(A, chunks, nchunks, gpair,
                                                                                    gcoef, s, E, Ew, US, sig);
}

void launch_residual_owner_df(cudaStream_t st, const OpView& A, bool offsets, const unsigned char* sig,
                              const float4* u, const float2* psi32, const float* Wh, const float* Wl, double2* r,
                              float2* b, float4* part_r, float4* part_b, const int* need_b, int* err)
{
    dim3 grid(A.nch, (A.n1 + TR - 1) / TR);
    const size_t sm = residual_own_df_smem();
    if (offsets) {
        k_residual_own_df<true, true><<<grid, NTHR_OWN, sm, st>>>(A, u, psi32, Wh, Wl, r, b, part_r, part_b, sig,
                                                                need_b, err);
        k_residual_own_df<false, true><<<grid, NTHR_OWN, sm, st>>>(A, u, psi32, Wh, Wl, r, b, part_r, part_b, sig,
                                                                 need_b, err);
    } else {
        k_residual_own_df<true, false><<<grid, NTHR_OWN, sm, st>>>(A, u, psi32, Wh, Wl, r, b, part_r, part_b, sig,
                                                                 need_b, err);
        k_residual_own_df<false, false><<<grid, NTHR_OWN, sm, st>>>(A, u, psi32, Wh, Wl, r, b, part_r, part_b, sig,
                                                                  need_b, err);
    }
}

int residual_sig_bytes() { return SIG_BYTES; }
size_t residual_us_floats(int nch, int n1) { return (size_t)nch * us_stride(n1); }

void launch_residual_gather_df(cudaStream_t st, const OpView& A, const float2* S, const float2* Ht, const float4* u,
                               const float4* v, const float2* psi32, double2* r, const float2* b,
                               const float4* part_r, const float4* part_b, const int* need_b, double* pn_r,
                               double* pn_b)
{
    dim3 grid(A.nch, (A.n1 + TR - 1) / TR);
    k_residual_gather_df<<<grid, NT, 0, st>>>(A, S, Ht, u, v, psi32, r, b, part_r, part_b, need_b, pn_r, pn_b);
}

size_t apply_own32_smem() { return (size_t)NST * STAGE32 * sizeof(float); }
int apply_own_tile() { return TR; }
int apply_own_nout() { return NOUT; }
bool apply_own_supported(const OpView& A) { return A.bd == BDO; }

// once per process and device before the first launch (and before any stream capture)
cudaError_t apply_own32_prepare()
{
    cudaError_t e =
        cudaFuncSetAttribute(k_apply_own32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_own32_smem());
    if (e != cudaSuccess) return e;
    const int sm = (int)residual_own_df_smem();
    if ((e = cudaFuncSetAttribute(k_residual_own_df<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_residual_own_df<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_residual_own_df<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) !=
            cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_residual_own_df<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

void launch_apply_own32(cudaStream_t st, const OpView& A, const float* S, const float* H, int sign, const void* x,
                        const float* W, void* y, float4* part, const void* bsub, const void* dv, double2* pdot,
                        double* pnrm, const KState* skip, int* err)
{
    dim3 grid(A.nch, (A.n1 + TR - 1) / TR);
    k_apply_own32<<<grid, 2 * NT + 32, apply_own32_smem(), st>>>(A, S, H, sign, (const float2*)x, W, (float2*)y, part,
                                                            skip, err);
    k_apply_gather32<<<grid, NT, 0, st>>>(A, sign, (float2*)y, part, (const float2*)bsub, (const float2*)dv, pdot,
                                          pnrm, skip);
}

}  // namespace dg
