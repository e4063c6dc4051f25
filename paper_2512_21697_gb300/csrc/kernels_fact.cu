// kernels_fact.cu -- the complex64 operator apply A_+- x of the inner solve in factorised form:
// the coupling values are never stored.
//
// The coupling block of a pair (a, b) is W_ab = sum_l cA_l K_l(ka, kb) + cB_l KT_l(kb, ka) with
// K_l(k', k) = G0 + k' G1 + k G2 + k' k G3 (the combined radial bands of Eq. fullH; G^n the
// time-dependent bands of multipole l) and KT the block transpose.  Grouping the monomials by the
// channel whose vector they multiply,
//   K_l(ka, kb) x_b         = U_l^b + ka V_l^b,    U = (G0 + kb G2) x_b,   V = (G1 + kb G3) x_b
//   blockT(K_l(kb, ka)) x_b = U'_l^b + ka V'_l^b,  U' = blockT(G0 + kb G1) x_b,  V' = blockT(G2 + kb G3) x_b
// so four band products per (channel, multipole) serve every partner of the channel, and the
// per-pair work is a short combination with the angular coefficients.  For the transposed use of
// a pair (rows of b from x_a), W_ab^T x_a = sum_l cA_l (U'_l^a + kb V'_l^a) + cB_l (U_l^a + kb V_l^a).
//
// Two passes per radial tile of FTR rows: k_fact_radial32 (block = a chunk of up to FCOL channels
// of one kappa, one multipole) forms the four products at the tile's rows, the bands built on the
// fly from G and shared by the chunk's channels; k_fact_angular32 (block = channel) combines its
// partners' products, adds the diagonal block and runs the BiCGSTAB epilogues.  The products of a
// tile (about 53 MB at the production size) stay in L2 between the two passes.
#include <cuda_runtime.h>

#include <cstdint>

#include "device.h"
#include "kernels.h"

namespace dg {

namespace {
constexpr int BDF = 13;          // block diagonals (order-7 splines)
constexpr int HF = (BDF - 1) / 2;

__device__ __forceinline__ bool used_f(int kappa, int slot, int type)
{
    return slot != 0 || (type == 0 ? kappa == -1 : kappa == 1);
}
}  // namespace

int fact_tile() { return FTR; }

// U, V, U', V' of the chunk's channels at rows r0 .. r0 + FTR - 1 for multipole blockIdx.y.
// Z[((ch * L + l) * 4 + beta) * FTR + lr][t], complex64.
__global__ void __launch_bounds__(2 * FTR) k_fact_radial32(OpView A, const RadChunk* __restrict__ rc,
                                                           const float2* __restrict__ G, int L,
                                                           const float2* __restrict__ x, float2* __restrict__ Z,
                                                           int tile, const KState* skip)
{
    if (skip && skip->done) return;   // uniform over the grid: the solve already finished
    __shared__ float2 xs[FCOL][FTR + 2 * HF][2];
    const RadChunk c = rc[blockIdx.x];
    const int l = blockIdx.y;
    const int n1 = A.n1;
    const int r0 = tile * FTR, rows = min(FTR, n1 - r0);
    const int64_t be = (int64_t)n1 * BDF * 4;   // entries of one band
    // the chunk's vector windows, rows r0 - h .. r0 + FTR + h; zero outside the grid and at unused
    // functions (the stored coupling would be zero there)
    for (int i = threadIdx.x; i < c.count * (FTR + 2 * HF) * 2; i += blockDim.x) {
        const int col = i / ((FTR + 2 * HF) * 2), rem = i - col * (FTR + 2 * HF) * 2;
        const int w = rem >> 1, u = rem & 1, rr = r0 - HF + w;
        const int ch = A.prec_order[c.first + col];
        float2 v = make_float2(0.f, 0.f);
        if (rr >= 0 && rr < n1 && used_f(c.kappa, rr, u)) v = x[((int64_t)ch * n1 + rr) * 2 + u];
        xs[col][w][u] = v;
    }
    __syncthreads();
    const int lr = threadIdx.x >> 1, t = threadIdx.x & 1, r = r0 + lr;
    if (lr >= rows) return;   // no barrier below
    const float kap = (float)c.kappa;
    const float2* Gl = G + (int64_t)l * 4 * be;
    for (int beta = 0; beta < 4; beta++) {
        // band entries of row (r, t): U (G0 + k G2), V (G1 + k G3) at (r, d, t, u); U', V' the
        // block transposes (G0 + k G1), (G2 + k G3) at (r + d - h, 2h - d, u, t)
        const int na = beta == 0 ? 0 : beta == 1 ? 1 : beta == 2 ? 0 : 2;
        const int nb = beta == 0 ? 2 : beta == 1 ? 3 : beta == 2 ? 1 : 3;
        float e[BDF][2];
#pragma unroll
        for (int d = 0; d < BDF; d++) {
            const int rr = r + d - HF;
            const bool inb = rr >= 0 && rr < n1;
#pragma unroll
            for (int u = 0; u < 2; u++) {
                float v = 0.f;
                if (inb) {
                    int64_t idx = beta < 2 ? (((int64_t)r * BDF + d) * 2 + t) * 2 + u
                                           : (((int64_t)rr * BDF + (2 * HF - d)) * 2 + u) * 2 + t;
                    v = fmaf(kap, Gl[nb * be + idx].x, Gl[na * be + idx].x);
                }
                e[d][u] = v;
            }
        }
        for (int col = 0; col < c.count; col++) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < BDF; d++) {
                const float2 x0 = xs[col][lr + d][0], x1 = xs[col][lr + d][1];
                acc.x = fmaf(e[d][0], x0.x, acc.x); acc.x = fmaf(e[d][1], x1.x, acc.x);
                acc.y = fmaf(e[d][0], x0.y, acc.y); acc.y = fmaf(e[d][1], x1.y, acc.y);
            }
            const int ch = A.prec_order[c.first + col];
            Z[((((int64_t)ch * L + l) * 4 + beta) * FTR + lr) * 2 + t] = acc;
        }
    }
}

// y_a = D^sign x_a - sign sum_own W_ab x_b + sign sum_in W_a'a^T x_a' at the tile's rows, from the
// tile's products; then y <- bsub - y, <dv, y> and ||y||^2 partials (slot tile * nch + a).
__global__ void __launch_bounds__(2 * FTR) k_fact_angular32(OpView A, const float* __restrict__ S,
                                                            const float* __restrict__ H, int sign,
                                                            const float2* __restrict__ x,
                                                            const float2* __restrict__ Z, int L,
                                                            const float4* __restrict__ cab, float2* __restrict__ y,
                                                            const float2* __restrict__ bsub,
                                                            const float2* __restrict__ dv, double2* part_dot,
                                                            double* part_nrm, int tile, const KState* skip)
{
    if (skip && skip->done) return;
    const int n1 = A.n1, a = blockIdx.x;
    const int r0 = tile * FTR, rows = min(FTR, n1 - r0);
    const int lr = threadIdx.x >> 1, t = threadIdx.x & 1, r = r0 + lr;
    const bool act = lr < rows;
    double2 dsum = make_double2(0, 0);
    double nsum = 0;
    if (act) {
        const int ka = A.ch_kappa[a];
        const float fka = (float)ka;
        // diagonal block (S + sign i tau H0) x_a, row (r, t)
        const int ks = A.ch_kslot[a];
        const float* Sk = S + ((int64_t)ks * n1 + r) * BDF * 4;
        const float* Hk = H + ((int64_t)ks * n1 + r) * BDF * 4;
        const float2* xa = x + (int64_t)a * 2 * n1;
        const float st = (float)(sign * A.tau);
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int d = 0; d < BDF; d++) {
            const int rr = r + d - HF;
            if (rr < 0 || rr >= n1) continue;
            for (int u = 0; u < 2; u++) {
                const float s = Sk[d * 4 + 2 * t + u], h = st * Hk[d * 4 + 2 * t + u];
                const float2 xv = xa[2 * rr + u];
                v.x += s * xv.x - h * xv.y;
                v.y += s * xv.y + h * xv.x;
            }
        }
        if (used_f(ka, r, t)) {
            // partners b of the pairs the channel owns: W_ab x_b
            float2 co = make_float2(0.f, 0.f), ci = make_float2(0.f, 0.f);
            for (int e = A.own_start[a]; e < A.own_start[a + 1]; e++) {
                const int64_t p = A.own_pair[e];
                const int b = A.own_nbr[e];
                for (int q = A.term_start[p]; q < A.term_start[p + 1]; q++) {
                    const int l = A.term_l[q];
                    const float4 cf = cab[q];   // (cA hi, cA lo, cB hi, cB lo)
                    const float2* zb = Z + (((int64_t)b * L + l) * 4 * FTR + lr) * 2 + t;
                    const float2 U = zb[0], V = zb[FTR * 2], Up = zb[2 * FTR * 2], Vp = zb[3 * FTR * 2];
                    co.x += cf.x * fmaf(fka, V.x, U.x) + cf.z * fmaf(fka, Vp.x, Up.x);
                    co.y += cf.x * fmaf(fka, V.y, U.y) + cf.z * fmaf(fka, Vp.y, Up.y);
                }
            }
            // lower channels a' of the pairs the channel is the upper channel of: W_a'a^T x_a'
            for (int e = A.in_start[a]; e < A.in_start[a + 1]; e++) {
                const int64_t p = A.in_pair[e];
                const int a2 = A.pair_a[p];
                for (int q = A.term_start[p]; q < A.term_start[p + 1]; q++) {
                    const int l = A.term_l[q];
                    const float4 cf = cab[q];
                    const float2* za = Z + (((int64_t)a2 * L + l) * 4 * FTR + lr) * 2 + t;
                    const float2 U = za[0], V = za[FTR * 2], Up = za[2 * FTR * 2], Vp = za[3 * FTR * 2];
                    ci.x += cf.x * fmaf(fka, Vp.x, Up.x) + cf.z * fmaf(fka, V.x, U.x);
                    ci.y += cf.x * fmaf(fka, Vp.y, Up.y) + cf.z * fmaf(fka, V.y, U.y);
                }
            }
            const float sg = (float)sign;
            v.x += sg * (ci.x - co.x);
            v.y += sg * (ci.y - co.y);
        }
        const int64_t o = ((int64_t)a * n1 + r) * 2 + t;
        if (bsub) {
            const float2 bb = bsub[o];
            v = make_float2(bb.x - v.x, bb.y - v.y);
        }
        y[o] = v;
        if (dv) {
            const float2 w = dv[o];
            dsum.x = (double)w.x * v.x + (double)w.y * v.y;
            dsum.y = (double)w.x * v.y - (double)w.y * v.x;
        }
        nsum = (double)v.x * v.x + (double)v.y * v.y;
    }
    if (part_dot || part_nrm)
        block_reduce_store(dsum, nsum, part_dot, part_nrm, (int64_t)tile * gridDim.x + blockIdx.x);
}

void launch_fact32(cudaStream_t st, const OpView& A, const RadChunk* rc, int nrc, const float2* G, int L,
                   const float* S, const float* H, int sign, const void* x, float2* Z, const float4* cab, void* y,
                   const void* bsub, const void* dv, double2* pdot, double* pnrm, const KState* skip)
{
    const int ntile = (A.n1 + FTR - 1) / FTR;
    for (int tile = 0; tile < ntile; tile++) {
        k_fact_radial32<<<dim3(nrc, L), 2 * FTR, 0, st>>>(A, rc, G, L, (const float2*)x, Z, tile, skip);
        k_fact_angular32<<<A.nch, 2 * FTR, 0, st>>>(A, S, H, sign, (const float2*)x, Z, L, cab, (float2*)y,
                                                     (const float2*)bsub, (const float2*)dv, pdot, pnrm, tile,
                                                     skip);
    }
}

}  // namespace dg
