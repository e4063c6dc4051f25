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
// Two passes per radial tile of FTR rows, the products of a tile (about 53 MB at the production
// size) staying in L2 between them.  Two forms:
//  - per-channel (mode 2): k_fact_radial32 (block = a chunk of up to FCOL channels of one kappa, one
//    multipole; a thread per row) forms the four products, the bands built on the fly from G and
//    shared by the chunk's channels; k_fact_angular32 (block = channel) reads each partner's products
//    from L2 and combines them.  Every (partner, multipole) product is read once per output channel
//    that uses it (about 12 GB of L2 reads per apply at the production size).
//  - subgroup (mode 1), one launch of k_fact_tile32 per tile: its radial blocks put up to FLANE
//    channels of one or two kappas on the lanes of a warp, each lane holding its channel's vector
//    window in registers and the band entries read as shared-memory broadcasts (eight FMAs per
//    16-byte load); its angular blocks (FSG output channels of one mu) load the union of their
//    (partner, multipole) products once and apply each to all FSG outputs from registers.  The
//    partners of a channel all have mu +- 1, so the outputs of one mu share them; ordered by the
//    parity of the orbital l and |kappa|, about half of the FSG coefficient sets of an item are
//    nonzero at the production size and each product is read about 3.5 times per apply instead of
//    30.  Launch t runs the angular blocks of tile t beside the radial blocks of tile t + 1 (two
//    product buffers): both kinds wait on memory far more than they compute, so the SMs interleave
//    them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "device.h"
#include "kernels.h"
#include "mbar.cuh"

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

void launch_fact32_chan(cudaStream_t st, const OpView& A, const RadChunk* rc, int nrc, const float2* G, int L,
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


// ---- subgroup form ---------------------------------------------------------------------------

namespace {
constexpr int RSL = 4;                        // radial slots per thread (radial pass)
constexpr int RWARP = 8;                      // warps per radial block: RWARP x RSL slots
constexpr int RSLOTS = RWARP * RSL;           // slots per radial block (half a tile)
constexpr int GROWS = RSLOTS + 2 * HF;        // rows of G (and of the vectors) the block's slots reach
constexpr int XW = GROWS + 1;                 // staged vector window stride (float4): conflict-free lanes
constexpr int OW = RSLOTS + 1;                // staged output stride (float4)
static_assert(FTR % RSLOTS == 0, "radial blocks tile the radial tile");
// dynamic shared memory of the radial pass, float4 entries: G^n rows [4][GROWS][BDF], later the
// vector windows [FLANE][XW] and then the outputs [FLANE][OW] in the same space; the combined bands
// of the block's two kappas [2][4][RSLOTS][BDF]
constexpr int RAD_G = 4 * GROWS * BDF, RAD_E = 4 * RSLOTS * BDF, RAD_X = FLANE * XW;
constexpr int RAD_GX = RAD_G > RAD_X ? RAD_G : RAD_X;
static_assert(FLANE * OW <= RAD_X, "the output staging fits in the vector staging");
// the second kappa's bands start one float4 past a 128-byte boundary, so that the two broadcast
// addresses of a warp holding two chunks fall in different banks
constexpr int RAD_E1 = RAD_E + 1;
constexpr size_t RAD_SMEM = (size_t)(RAD_GX + RAD_E1 + RAD_E) * sizeof(float4);

constexpr int FSPLIT = 4;                     // threads per slot in the angular pass (items split)
constexpr int FPIPE = 4;                      // items each thread has in flight
static_assert(FSG % FSPLIT == 0, "outputs split evenly over the item splits");
}  // namespace

// U, V, U', V' at the RSLOTS slots of block (pack, l, part) of the tile.  A pack is one or two kappa
// chunks whose channels together fill at most the FLANE lanes of a warp.  The block stages, with
// asynchronous copies all in flight at once, the hi words of the four G^n bands of multipole l at the
// rows its slots reach, and forms the four combined bands of each chunk's kappa at its slots,
// es[chunk][beta][slot][d]; then it stages the channels' vector windows (in the space the bands came
// through).  Lane = channel: each thread takes RSL consecutive slots of its channel and both function
// types, with its window in registers; the lanes of a chunk read the same band entry (a broadcast;
// two addresses per warp when it holds two chunks), eight FMAs per 16-byte load.  The products go
// out through shared memory so that the stores of a channel's rows are coalesced.
__device__ __forceinline__ void fact_radial_block(const OpView& A, const RadPack* __restrict__ rp,
                                                  const float* __restrict__ Gh, int L, const float2* __restrict__ x,
                                                  float2* __restrict__ Z, int tile, int pack, int l, int part,
                                                  float4* rsm, int* s_ch, int* s_kap)
{
    float4* Gs = rsm;                  // [n][row][d]; later [lane][XW] windows, then [lane][OW] outputs
    float4* xs = rsm;
    float4* es = rsm + RAD_GX;         // [chunk][beta][slot][d], chunk stride RAD_E1
    const RadPack* pk = rp + pack;
    const int n0 = pk->c[0].count, n1c = pk->c[1].count, nl = n0 + n1c;   // lanes of chunk 0, lanes in use
    const int n1 = A.n1;
    const int ls0 = part * RSLOTS;             // first slot of the block within the tile
    const int s0 = tile * FTR + ls0;           // its global slot
    // G^n at rows s0 - h .. s0 + RSLOTS - 1 + h (zero outside the grid): per n a contiguous range of
    // GROWS rows, BDF float4 (one 2 x 2 block per diagonal) each
    const float4* Gl = reinterpret_cast<const float4*>(Gh) + (int64_t)l * 4 * n1 * BDF;
    for (int n = 0; n < 4; n++) {
        for (int i = threadIdx.x; i < GROWS * BDF; i += blockDim.x) {
            const int rr = s0 - HF + i / BDF;
            const bool in = rr >= 0 && rr < n1;
            cp_async16z(&Gs[n * GROWS * BDF + i], Gl + ((int64_t)n * n1 + (in ? rr : 0)) * BDF + i % BDF,
                        in ? 16u : 0u);
        }
    }
    if (threadIdx.x < FLANE) {
        const int ln = threadIdx.x, k = ln < n0 ? 0 : 1;
        s_ch[ln] = ln < nl ? A.prec_order[pk->c[k].first + ln - (k ? n0 : 0)] : 0;
        s_kap[ln] = pk->c[k].kappa;
    }
    cp_async_wait_all();
    __syncthreads();
    // combined bands of each chunk's kappa: U (G0 + k G2), V (G1 + k G3) at (r, d, t, u); U', V' the
    // block transposes (G0 + k G1), (G2 + k G3) at (r + d - h, 2h - d, u, t); zero where the row or
    // the column is outside the grid.  Thread -> (beta, slot, half of the diagonals).
    {
        static_assert(RWARP * 32 == 8 * RSLOTS, "one thread per (beta, slot, half)");
        const int ls = threadIdx.x % RSLOTS, beta = (threadIdx.x / RSLOTS) & 3, dh = threadIdx.x / (4 * RSLOTS);
        const int na = beta == 0 ? 0 : beta == 1 ? 1 : beta == 2 ? 0 : 2;
        const int nb = beta == 0 ? 2 : beta == 1 ? 3 : beta == 2 ? 1 : 3;
        const int r = s0 + ls;
        for (int k = 0; k < (n1c ? 2 : 1); k++) {
            const float kap = (float)pk->c[k].kappa;
            for (int d = dh * 7; d < min(BDF, dh * 7 + 7); d++) {
                const int rr = r + d - HF;
                float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r < n1 && rr >= 0 && rr < n1) {
                    // Gs row of slot r is ls + h; of column slot rr, ls + d
                    const int row = beta < 2 ? ls + HF : ls + d, dd = beta < 2 ? d : 2 * HF - d;
                    const float4 ga = Gs[(na * GROWS + row) * BDF + dd], gb = Gs[(nb * GROWS + row) * BDF + dd];
                    e = make_float4(fmaf(kap, gb.x, ga.x), fmaf(kap, gb.y, ga.y), fmaf(kap, gb.z, ga.z),
                                    fmaf(kap, gb.w, ga.w));
                    if (beta >= 2) e = make_float4(e.x, e.z, e.y, e.w);   // (u, t) -> (t, u)
                }
                es[k * RAD_E1 + (beta * RSLOTS + ls) * BDF + d] = e;
            }
        }
    }
    __syncthreads();   // the G rows are no longer needed: their space takes the vector windows
    // the channels' vector windows, slots s0 - h .. s0 + RSLOTS - 1 + h, both types (zero outside the
    // grid; the unused functions are masked when the windows are read)
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (int i = threadIdx.x; i < nl * GROWS; i += blockDim.x) {
        const int cc = i / GROWS, j = i - cc * GROWS, rr = s0 - HF + j;
        const bool in = rr >= 0 && rr < n1;
        cp_async16z(&xs[cc * XW + j], x4 + (int64_t)s_ch[cc] * n1 + (in ? rr : 0), in ? 16u : 0u);
    }
    cp_async_wait_all();
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool act = lane < nl;
    const int kap = s_kap[lane];
    const int sw = s0 + w * RSL;   // the thread's first slot
    float4 xw[RSL + 2 * HF];       // the thread's window: (x0.re, x0.im, x1.re, x1.im)
#pragma unroll
    for (int j = 0; j < RSL + 2 * HF; j++) {
        float4 v = act ? xs[lane * XW + w * RSL + j] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int rr = sw - HF + j;
        if (!used_f(kap, rr, 0)) { v.x = 0.f; v.y = 0.f; }   // only slot 0 can be unused
        if (!used_f(kap, rr, 1)) { v.z = 0.f; v.w = 0.f; }
        xw[j] = v;
    }
    __syncthreads();   // xs is free: it takes the outputs from here on
    float4* Z4 = reinterpret_cast<float4*>(Z);
    const float4* ek = es + (lane < n0 ? 0 : RAD_E1);
#pragma unroll 1
    for (int beta = 0; beta < 4; beta++) {
        if (act) {
            float4 acc[RSL];   // (row t = 0 complex, row t = 1 complex)
#pragma unroll
            for (int s = 0; s < RSL; s++) acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4* eb = ek + (beta * RSLOTS + w * RSL) * BDF;
#pragma unroll
            for (int s = 0; s < RSL; s++) {
#pragma unroll
                for (int d = 0; d < BDF; d++) {
                    const float4 e = eb[s * BDF + d];
                    const float4 xv = xw[s + d];
                    acc[s].x = fmaf(e.x, xv.x, fmaf(e.y, xv.z, acc[s].x));
                    acc[s].y = fmaf(e.x, xv.y, fmaf(e.y, xv.w, acc[s].y));
                    acc[s].z = fmaf(e.z, xv.x, fmaf(e.w, xv.z, acc[s].z));
                    acc[s].w = fmaf(e.z, xv.y, fmaf(e.w, xv.w, acc[s].w));
                }
            }
#pragma unroll
            for (int s = 0; s < RSL; s++) xs[lane * OW + w * RSL + s] = acc[s];
        }
        __syncthreads();
        // rows ls0 .. ls0 + RSLOTS - 1 of (channel, l, beta): RSLOTS consecutive float4 per channel
        for (int i = threadIdx.x; i < nl * RSLOTS; i += blockDim.x) {
            const int cc = i / RSLOTS, j = i - cc * RSLOTS;
            Z4[(((int64_t)s_ch[cc] * L + l) * 4 + beta) * FTR + ls0 + j] = xs[cc * OW + j];
        }
        __syncthreads();
    }
}

// Outputs of subgroup sub at the tile's rows: y_a = D^sign x_a + sign sum_items coef . products,
// then y <- bsub - y and the <dv, y>, ||y||^2 partials (slot tile * nsub + subgroup).  The block first
// copies its items' coefficient sets (FSG float4 each) and offsets into shared memory.  Thread
// (split grp, slot ls) takes items grp, grp + FSPLIT, ... with FPIPE of them in flight: the four
// products of an item at its slot (both types, 64 bytes) are loaded FPIPE items ahead of their use,
// so each thread keeps 256 bytes of loads outstanding.  The splits' sums meet in shared memory in a
// fixed order.
__device__ __forceinline__ void fact_mu_block(const OpView& A, const float* __restrict__ ST,
                                              const float* __restrict__ HT, int sign, const float2* __restrict__ x,
                                              const float2* __restrict__ Z, const FactSub* __restrict__ subs,
                                              const int* __restrict__ item_off, const float4* __restrict__ item_coef,
                                              float2* __restrict__ y, const float2* __restrict__ bsub,
                                              const float2* __restrict__ dv, double2* part_dot, double* part_nrm,
                                              int tile, int sub, int nsub, float4* msm)
{
    float4* red = msm;                                              // [split][FSG][FTR]
    const int tid = threadIdx.x;
    const int gfirst = subs[sub].first, gcount = subs[sub].count;
    float4* s_coef = msm + FSPLIT * FSG * FTR;                      // [item][FSG]
    int* s_off = reinterpret_cast<int*>(s_coef + (size_t)gcount * FSG);  // [item]
    for (int k = tid; k < gcount * FSG; k += blockDim.x) cp_async16z(&s_coef[k], item_coef + (int64_t)gfirst * FSG + k, 16u);
    for (int k = tid; k < gcount; k += blockDim.x) s_off[k] = item_off[gfirst + k];
    cp_async_wait_all();
    __syncthreads();
    const int ls = tid % FTR, grp = tid / FTR;
    float4 acc[FSG];
#pragma unroll
    for (int j = 0; j < FSG; j++) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4* Zt = reinterpret_cast<const float4*>(Z) + ls;
    float4 B[FPIPE][4];   // the products of the items in flight: (U, V, U', V') at the thread's slot
#pragma unroll
    for (int q = 0; q < FPIPE; q++) {
        const int k = grp + q * FSPLIT;
        if (k < gcount) {
            const float4* z = Zt + (int64_t)s_off[k] * 4 * FTR;
#pragma unroll
            for (int b = 0; b < 4; b++) B[q][b] = __ldcg(z + b * FTR);
        }
    }
    for (int k0 = grp; k0 < gcount; k0 += FPIPE * FSPLIT) {
#pragma unroll
        for (int q = 0; q < FPIPE; q++) {
            const int k = k0 + q * FSPLIT;
            if (k < gcount) {
                const float4 U = B[q][0], V = B[q][1], Up = B[q][2], Vp = B[q][3];
                const int kn = k + FPIPE * FSPLIT;   // refill the slot with the item FPIPE rounds ahead
                if (kn < gcount) {
                    const float4* z = Zt + (int64_t)s_off[kn] * 4 * FTR;
#pragma unroll
                    for (int b = 0; b < 4; b++) B[q][b] = __ldcg(z + b * FTR);
                }
                const float4* cf = s_coef + (int64_t)k * FSG;
#pragma unroll
                for (int j = 0; j < FSG; j++) {
                    const float4 c = cf[j];   // the same address in every thread: a broadcast
                    acc[j].x = fmaf(c.x, U.x, fmaf(c.y, V.x, fmaf(c.z, Up.x, fmaf(c.w, Vp.x, acc[j].x))));
                    acc[j].y = fmaf(c.x, U.y, fmaf(c.y, V.y, fmaf(c.z, Up.y, fmaf(c.w, Vp.y, acc[j].y))));
                    acc[j].z = fmaf(c.x, U.z, fmaf(c.y, V.z, fmaf(c.z, Up.z, fmaf(c.w, Vp.z, acc[j].z))));
                    acc[j].w = fmaf(c.x, U.w, fmaf(c.y, V.w, fmaf(c.z, Up.w, fmaf(c.w, Vp.w, acc[j].w))));
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < FSG; j++) red[(grp * FSG + j) * FTR + ls] = acc[j];
    __syncthreads();
    const int n1 = A.n1, r = tile * FTR + ls;
    double2 dsum = make_double2(0, 0);
    double nsum = 0;
    if (r < n1) {
        const float st = (float)(sign * A.tau), sg = (float)sign;
#pragma unroll 1
        for (int j = grp; j < FSG; j += FSPLIT) {
            const int a = subs[sub].out[j];
            if (a < 0) continue;
            float4 cs = red[j * FTR + ls];
#pragma unroll
            for (int q = 1; q < FSPLIT; q++) {
                const float4 o = red[(q * FSG + j) * FTR + ls];
                cs.x += o.x; cs.y += o.y; cs.z += o.z; cs.w += o.w;
            }
            const int ka = A.ch_kappa[a], ks = A.ch_kslot[a];
            if (!used_f(ka, r, 0)) { cs.x = 0.f; cs.y = 0.f; }   // the coupling is zero at unused rows
            if (!used_f(ka, r, 1)) { cs.z = 0.f; cs.w = 0.f; }
            // diagonal block (S + sign i tau H0) x_a; bands with the rows innermost: diagonal d of row
            // r is the float4 at (ks BDF + d) n1 + r
            const float4* Sk = reinterpret_cast<const float4*>(ST) + (int64_t)ks * BDF * n1 + r;
            const float4* Hk = reinterpret_cast<const float4*>(HT) + (int64_t)ks * BDF * n1 + r;
            const float4* xa = reinterpret_cast<const float4*>(x) + (int64_t)a * n1;
            float2 d0 = make_float2(0.f, 0.f), d1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < BDF; d++) {
                const int rr = r + d - HF;
                if (rr < 0 || rr >= n1) continue;
                const float4 xv = xa[rr], sv = Sk[(int64_t)d * n1], hv = Hk[(int64_t)d * n1];
                const float h00 = st * hv.x, h01 = st * hv.y, h10 = st * hv.z, h11 = st * hv.w;
                d0.x += sv.x * xv.x + sv.y * xv.z - (h00 * xv.y + h01 * xv.w);
                d0.y += sv.x * xv.y + sv.y * xv.w + (h00 * xv.x + h01 * xv.z);
                d1.x += sv.z * xv.x + sv.w * xv.z - (h10 * xv.y + h11 * xv.w);
                d1.y += sv.z * xv.y + sv.w * xv.w + (h10 * xv.x + h11 * xv.z);
            }
            float4 v = make_float4(d0.x + sg * cs.x, d0.y + sg * cs.y, d1.x + sg * cs.z, d1.y + sg * cs.w);
            const int64_t o = (int64_t)a * n1 + r;
            if (bsub) {
                const float4 bb = reinterpret_cast<const float4*>(bsub)[o];
                v = make_float4(bb.x - v.x, bb.y - v.y, bb.z - v.z, bb.w - v.w);
            }
            reinterpret_cast<float4*>(y)[o] = v;
            if (dv) {
                const float4 wv = reinterpret_cast<const float4*>(dv)[o];
                dsum.x += (double)wv.x * v.x + (double)wv.y * v.y + (double)wv.z * v.z + (double)wv.w * v.w;
                dsum.y += (double)wv.x * v.y - (double)wv.y * v.x + (double)wv.z * v.w - (double)wv.w * v.z;
            }
            nsum += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
        }
    }
    if (part_dot || part_nrm)
        block_reduce_store(dsum, nsum, part_dot, part_nrm, (int64_t)tile * nsub + sub);
}

// One launch per radial tile t = -1 .. ntile - 1: blocks 0 .. nsub_t - 1 run the angular pass of tile
// t (products in Z[t mod 2]), the others the radial pass of tile t + 1 (into Z[(t + 1) mod 2]).  The
// two passes are latency-bound with little issue pressure, so the SMs interleave them; the launch
// boundary orders each tile's products before their readers, and the products of tile t - 1 (read
// in launch t - 1) before they are overwritten by launch t.  Angular blocks come first (the longer
// ones, heaviest subgroups first).
__global__ void __launch_bounds__(RWARP * 32, 2) k_fact_tile32(OpView A, const RadPack* __restrict__ rp, int nrp,
                                                              const FactSub* __restrict__ subs, int nsub, int nsub_t,
                                                              const int* __restrict__ item_off,
                                                              const float4* __restrict__ item_coef,
                                                              const float* __restrict__ Gh, int L,
                                                              const float* __restrict__ ST, const float* __restrict__ HT,
                                                              int sign, const float2* __restrict__ x,
                                                              const float2* __restrict__ Za, float2* __restrict__ Zr,
                                                              float2* __restrict__ y, const float2* __restrict__ bsub,
                                                              const float2* __restrict__ dv, double2* part_dot,
                                                              double* part_nrm, int tile, const KState* skip)
{
    static_assert(RWARP * 32 == FTR * FSPLIT, "both passes run 256-thread blocks");
    if (skip && skip->done) return;   // uniform over the grid: the solve already finished
    extern __shared__ float4 fsm[];
    __shared__ int s_ch[FLANE], s_kap[FLANE];
    const int b = blockIdx.x;
    if (b < nsub_t) {
        fact_mu_block(A, ST, HT, sign, x, Za, subs, item_off, item_coef, y, bsub, dv, part_dot, part_nrm, tile, b,
                      nsub, fsm);
    } else {
        const int rb = b - nsub_t;   // (pack, l, part) with part fastest
        const int part = rb % (FTR / RSLOTS), l = (rb / (FTR / RSLOTS)) % L, pack = rb / ((FTR / RSLOTS) * L);
        if (pack < nrp) fact_radial_block(A, rp, Gh, L, x, Zr, tile + 1, pack, l, part, fsm, s_ch, s_kap);
    }
}

// dynamic shared memory of the merged pass: the larger of the radial pass's staging and the angular
// pass's reduction, coefficient sets and offsets (subgroups of at most n items)
static size_t tile_smem(int n)
{
    const size_t mu = (size_t)FSPLIT * FSG * FTR * sizeof(float4) + (size_t)n * (FSG * sizeof(float4) + sizeof(int));
    return std::max(RAD_SMEM, mu);
}

// The limit only grows: an operator with fewer items per subgroup must not lower the limit that a
// larger operator of the same process launches with.
cudaError_t fact_sub_prepare(int max_items)
{
    static std::mutex mu;
    static size_t limit = 0;
    std::lock_guard<std::mutex> lock(mu);
    limit = std::max(limit, tile_smem(max_items));
    return cudaFuncSetAttribute(k_fact_tile32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
}

// Z holds two tiles' products (2 x channels x multipoles x 4 x FTR x 2 complex64)
void launch_fact32_sub(cudaStream_t st, const OpView& A, const RadPack* rl, int nrl, const FactSub* subs, int nsub,
                       int max_items, const int* item_off, const float4* item_coef, const float* Gh, int L,
                       const float* ST, const float* HT, int sign, const void* x, float2* Z, void* y,
                       const void* bsub, const void* dv, double2* pdot, double* pnrm, const KState* skip)
{
    const int ntile = (A.n1 + FTR - 1) / FTR;
    const int nrad = nrl * L * (FTR / RSLOTS);
    const size_t zhalf = (size_t)A.nch * L * 4 * FTR * 2;   // float2 per tile buffer
    const size_t smem = tile_smem(max_items);
    for (int t = -1; t < ntile; t++) {
        const int nsub_t = t >= 0 ? nsub : 0;
        const int nrad_t = t + 1 < ntile ? nrad : 0;
        float2* Za = Z + (size_t)((t + 2) % 2) * zhalf;
        float2* Zr = Z + (size_t)((t + 1) % 2) * zhalf;
        k_fact_tile32<<<nsub_t + nrad_t, RWARP * 32, smem, st>>>(A, rl, nrl, subs, nsub, nsub_t, item_off, item_coef,
                                                                 Gh, L, ST, HT, sign, (const float2*)x, Za, Zr,
                                                                 (float2*)y, (const float2*)bsub, (const float2*)dv,
                                                                 pdot, pnrm, t, skip);
    }
}

}  // namespace dg
