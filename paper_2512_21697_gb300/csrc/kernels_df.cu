// kernels_df.cu -- double-float (FP32-pair) kernels for the double-precision-accurate parts of the
// mixed-precision step: pulse bands, combined radial bands K_l(k', k), coupling assembly and the
// operator apply A_+- x with the residual epilogue b - A x (Eq. solPsi, Eq. fullH).  Values are
// stored as hi/lo float pairs; see df64.cuh for the arithmetic.
#include <cuda_runtime.h>

#include <algorithm>

#include "device.h"
#include "df64.cuh"
#include "kernels.h"

namespace dg {

__device__ __forceinline__ bool used_fn_df(int kappa, int slot, int type)
{
    return slot != 0 || (type == 0 ? kappa == -1 : kappa == 1);
}

// complex128 vector -> (re_hi, re_lo, im_hi, im_lo)
__global__ void k_split_vec(int64_t n, const double2* __restrict__ x, float4* __restrict__ xd)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 v = x[i];
    float2 a = df_split(v.x), b = df_split(v.y);
    xd[i] = make_float4(a.x, a.y, b.x, b.y);
}

// G[l][n][e] = sum_c s[l][c] M[l][c][n][e] in double, stored split (a few MB per step)
__global__ void k_field_combine_df(PulseView P, int block_elems, const double* s, float2* G, float* Gh)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int ln = blockIdx.y;
    if (e >= block_elems) return;
    int l = ln / 4, n = ln % 4;
    double v = 0;
    for (int c = 0; c < 3; c++) v += s[l * 3 + c] * P.M[(((int64_t)l * 3 + c) * 4 + n) * block_elems + e];
    const float2 g = df_split(v);
    G[(int64_t)ln * block_elems + e] = g;
    if (Gh) Gh[(int64_t)ln * block_elems + e] = g.x;   // the hi words alone, for the factorised apply
}

// K[key][e] = sum_n m_n G^n_l[e] and its block transpose KT[key][r][d][t][u] = K[key][r'][2h-d][u][t]
// (r' = r + d - h; zero where r' leaves the box), so that the assembly reads both the direct and the
// transposed term of a pair at the same coalesced position.  The monomials 1, k', k, k'k are
// integers, exact in FP32; G is a few MB and stays in L2, which serves the scattered reads of KT.
__global__ void k_build_K_df(OpView A, int block_elems, const float2* __restrict__ G, float2* __restrict__ K,
                             float2* __restrict__ KT)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= block_elems) return;
    int bd4 = A.bd * 4;
    int r = e / bd4, rem = e - r * bd4, d = rem >> 2, t = (rem >> 1) & 1, u = rem & 1;
    int rr = r + d - A.half;
    bool inb = rr >= 0 && rr < A.n1;
    int et = inb ? ((rr * A.bd + (2 * A.half - d)) * 2 + u) * 2 + t : 0;
    for (int key = blockIdx.y; key < A.nkeys; key += gridDim.y) {
        const double* m = A.key_mono + (int64_t)key * 4;
        const float2* Gl = G + (int64_t)A.key_l[key] * 4 * block_elems;
        DfAcc acc, act;
        df_zero(acc);
        df_zero(act);
        for (int n = 0; n < 4; n++) {
            float mn = (float)m[n];
            float2 g = Gl[(int64_t)n * block_elems + e];
            df_fma(acc, mn, 0.f, g.x, g.y);
            if (inb) {
                float2 gt = Gl[(int64_t)n * block_elems + et];
                df_fma(act, mn, 0.f, gt.x, gt.y);
            }
        }
        float h = acc.s + acc.c, ht = act.s + act.c;
        K[(int64_t)key * block_elems + e] = make_float2(h, (acc.s - h) + acc.c);
        KT[(int64_t)key * block_elems + e] = make_float2(ht, (act.s - ht) + act.c);
    }
}

// W_ab[r][d] = sum_terms cA K_l(ka,kb)[r][d] + cB KT_l(kb,ka)[r][d] in double-float; hi words to Wh
// (also the FP32 coupling values of the inner solve), lo words to Wl.  One thread per (radial row,
// block diagonal) of a pair: consecutive threads read and write consecutive 32-byte blocks.  Pairs
// sharing their kappa pair (all mu) are adjacent in the pair order, so their K bands come from L2.
template <int BD>
__global__ void __launch_bounds__(128) k_assemble_df(OpView A, const float2* __restrict__ K,
                                                     const float2* __restrict__ KT, const float4* __restrict__ cab,
                                                     float* __restrict__ Wh, float* __restrict__ Wl)
{
    const int bd = BD > 0 ? BD : A.bd;
    const int half = (bd - 1) / 2;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    int nrd = A.n1 * bd;
    if (idx >= nrd) return;
    int r = idx / bd, d = idx - r * bd, rr = r + d - half;
    bool inb = rr >= 0 && rr < A.n1;
    int64_t nb = (int64_t)nrd * 4;
    for (int64_t pi = blockIdx.y; pi < A.npairs; pi += gridDim.y) {
        int64_t p = A.pair_order[pi];
        DfAcc w[4];
        for (int k = 0; k < 4; k++) df_zero(w[k]);
        if (inb) {
            int q0 = A.term_start[p], q1 = A.term_start[p + 1];
            for (int q = q0; q < q1; q++) {
                float4 cf = cab[q];   // (cA hi, cA lo, cB hi, cB lo)
                const float4* g = reinterpret_cast<const float4*>(K + A.term_kd[q] * nb + (int64_t)idx * 4);
                const float4* gt = reinterpret_cast<const float4*>(KT + A.term_kt[q] * nb + (int64_t)idx * 4);
                float4 g01 = g[0], g23 = g[1], h01 = gt[0], h23 = gt[1];
                df_fma(w[0], cf.x, cf.y, g01.x, g01.y); df_fma(w[0], cf.z, cf.w, h01.x, h01.y);
                df_fma(w[1], cf.x, cf.y, g01.z, g01.w); df_fma(w[1], cf.z, cf.w, h01.z, h01.w);
                df_fma(w[2], cf.x, cf.y, g23.x, g23.y); df_fma(w[2], cf.z, cf.w, h23.x, h23.y);
                df_fma(w[3], cf.x, cf.y, g23.z, g23.w); df_fma(w[3], cf.z, cf.w, h23.z, h23.w);
            }
            int ka = A.ch_kappa[A.pair_a[p]], kb = A.ch_kappa[A.pair_b[p]];
            for (int k = 0; k < 4; k++) {
                int t = k / 2, u = k % 2;
                if (!used_fn_df(ka, r, t) || !used_fn_df(kb, rr, u)) df_zero(w[k]);
            }
        }
        int64_t o = (p * nrd + idx) * 4;
        float hh[4], ll[4];
        for (int k = 0; k < 4; k++) {
            hh[k] = w[k].s + w[k].c;
            ll[k] = (w[k].s - hh[k]) + w[k].c;
        }
        *reinterpret_cast<float4*>(Wh + o) = make_float4(hh[0], hh[1], hh[2], hh[3]);
        *reinterpret_cast<float4*>(Wl + o) = make_float4(ll[0], ll[1], ll[2], ll[3]);
    }
}

void launch_assemble_df(dim3 grid, cudaStream_t st, const OpView& A, const float2* K, const float2* KT,
                        const float4* cab, float* Wh, float* Wl)
{
    if (A.bd == 13) k_assemble_df<13><<<grid, 128, 0, st>>>(A, K, KT, cab, Wh, Wl);
    else k_assemble_df<0><<<grid, 128, 0, st>>>(A, K, KT, cab, Wh, Wl);
}

// Grouped form of the same assembly.  The pairs of one (kappa_a, kappa_b) group (all mu) combine
// the same K_l(ka, kb) and KT_l(kb, ka) bands with their own angular coefficients, so a block
// takes 128 (radial row, block diagonal) positions of one chunk of a group, forms the group's
// bands at its positions from G (as k_build_K_df: K = sum_n m_n G^n_l with m = 1, k', k, k'k,
// rounded to double-float; KT from the block-transposed position) and keeps them in registers,
// then writes the coupling values of every pair of the chunk.  G is a few MB and stays in L2; the
// combined bands are never stored.  Each pair's sum runs over the group's multipoles in
// increasing l, direct band first, as k_assemble_df; a multipole the pair lacks has zero
// coefficients.  NL = multipoles of the group (1..ASM_MAX_NL).
__device__ __forceinline__ float4 df_round2(const DfAcc& a, const DfAcc& b)
{
    float ha = a.s + a.c, hb = b.s + b.c;
    return make_float4(ha, (a.s - ha) + a.c, hb, (b.s - hb) + b.c);
}

template <int BD, int NL>
__device__ __forceinline__ void assemble_grp_body(const OpView& A, const AsmChunk& ch, const int* sp,
                                                  const float4* sc, int idx, const float2* __restrict__ G,
                                                  float* __restrict__ Wh, float* __restrict__ Wl)
{
    const int bd = BD > 0 ? BD : A.bd;
    const int half = (bd - 1) / 2;
    const int nrd = A.n1 * bd;
    const int64_t be = (int64_t)nrd * 4;   // elements of one band
    int r = idx / bd, d = idx - r * bd, rr = r + d - half;
    bool inb = rr >= 0 && rr < A.n1;
    bool keep[4];
    for (int k = 0; k < 4; k++)
        keep[k] = inb && used_fn_df(ch.ka, r, k / 2) && used_fn_df(ch.kb, rr, k % 2);
    const int idxt = inb ? rr * bd + (2 * half - d) : 0;   // block-transposed position
    const float mk[4] = {1.f, (float)ch.ka, (float)ch.kb, (float)(ch.ka * ch.kb)};
    const float mt[4] = {1.f, (float)ch.kb, (float)ch.ka, (float)(ch.ka * ch.kb)};
    float4 g[NL][2], h[NL][2];   // (hi, lo) pairs of the 4 block entries, direct and transposed band
#pragma unroll
    for (int j = 0; j < NL; j++) {
        const float4* Gl = reinterpret_cast<const float4*>(G + (int64_t)ch.l[j] * 4 * be);
        DfAcc kd[4], kt[4];
        for (int k = 0; k < 4; k++) { df_zero(kd[k]); df_zero(kt[k]); }
        for (int n = 0; n < 4; n++) {
            const float4* Gn = Gl + n * be / 2;
            float4 a0 = Gn[2 * idx], a1 = Gn[2 * idx + 1];   // entries (0,0), (0,1) | (1,0), (1,1)
            df_fma(kd[0], mk[n], 0.f, a0.x, a0.y);
            df_fma(kd[1], mk[n], 0.f, a0.z, a0.w);
            df_fma(kd[2], mk[n], 0.f, a1.x, a1.y);
            df_fma(kd[3], mk[n], 0.f, a1.z, a1.w);
            if (inb) {   // KT[t][u] = K[u][t] at the transposed position
                float4 b0 = Gn[2 * idxt], b1 = Gn[2 * idxt + 1];
                df_fma(kt[0], mt[n], 0.f, b0.x, b0.y);
                df_fma(kt[1], mt[n], 0.f, b1.x, b1.y);
                df_fma(kt[2], mt[n], 0.f, b0.z, b0.w);
                df_fma(kt[3], mt[n], 0.f, b1.z, b1.w);
            }
        }
        g[j][0] = df_round2(kd[0], kd[1]);
        g[j][1] = df_round2(kd[2], kd[3]);
        h[j][0] = df_round2(kt[0], kt[1]);
        h[j][1] = df_round2(kt[2], kt[3]);
    }
    for (int q = 0; q < ch.count; q++) {
        int64_t p = sp[q];
        DfAcc w[4];
        float4 cf = sc[q * ASM_MAX_NL];   // (cA hi, cA lo, cB hi, cB lo)
        df_mul(w[0], cf.x, cf.y, g[0][0].x, g[0][0].y); df_fma(w[0], cf.z, cf.w, h[0][0].x, h[0][0].y);
        df_mul(w[1], cf.x, cf.y, g[0][0].z, g[0][0].w); df_fma(w[1], cf.z, cf.w, h[0][0].z, h[0][0].w);
        df_mul(w[2], cf.x, cf.y, g[0][1].x, g[0][1].y); df_fma(w[2], cf.z, cf.w, h[0][1].x, h[0][1].y);
        df_mul(w[3], cf.x, cf.y, g[0][1].z, g[0][1].w); df_fma(w[3], cf.z, cf.w, h[0][1].z, h[0][1].w);
#pragma unroll
        for (int j = 1; j < NL; j++) {
            cf = sc[q * ASM_MAX_NL + j];
            df_fma(w[0], cf.x, cf.y, g[j][0].x, g[j][0].y); df_fma(w[0], cf.z, cf.w, h[j][0].x, h[j][0].y);
            df_fma(w[1], cf.x, cf.y, g[j][0].z, g[j][0].w); df_fma(w[1], cf.z, cf.w, h[j][0].z, h[j][0].w);
            df_fma(w[2], cf.x, cf.y, g[j][1].x, g[j][1].y); df_fma(w[2], cf.z, cf.w, h[j][1].x, h[j][1].y);
            df_fma(w[3], cf.x, cf.y, g[j][1].z, g[j][1].w); df_fma(w[3], cf.z, cf.w, h[j][1].z, h[j][1].w);
        }
        float hh[4], ll[4];
        for (int k = 0; k < 4; k++) {
            if (!keep[k]) df_zero(w[k]);
            hh[k] = w[k].s + w[k].c;
            ll[k] = (w[k].s - hh[k]) + w[k].c;
        }
        int64_t o = (p * nrd + idx) * 4;
        if (!DG_INB(A, o + 4 <= A.nb_coup, 4)) continue;
        *reinterpret_cast<float4*>(Wh + o) = make_float4(hh[0], hh[1], hh[2], hh[3]);
        *reinterpret_cast<float4*>(Wl + o) = make_float4(ll[0], ll[1], ll[2], ll[3]);
    }
}

template <int BD>
__global__ void __launch_bounds__(128) k_assemble_grp_df(OpView A, const AsmChunk* __restrict__ chunks, int nchunks,
                                                         const int* __restrict__ gpair,
                                                         const float4* __restrict__ gcoef,
                                                         const float2* __restrict__ G, float* __restrict__ Wh,
                                                         float* __restrict__ Wl)
{
    __shared__ int sp[ASM_CHUNK];
    __shared__ float4 sc[ASM_CHUNK * ASM_MAX_NL];
    const int bd = BD > 0 ? BD : A.bd;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = idx < A.n1 * bd;
    for (int c = blockIdx.y; c < nchunks; c += gridDim.y) {
        const AsmChunk ch = chunks[c];
        __syncthreads();   // the previous chunk's coefficients are no longer read
        for (int i = threadIdx.x; i < ch.count; i += blockDim.x) sp[i] = gpair[ch.first + i];
        for (int i = threadIdx.x; i < ch.count * ASM_MAX_NL; i += blockDim.x)
            sc[i] = gcoef[(int64_t)ch.first * ASM_MAX_NL + i];
        __syncthreads();
        if (!act) continue;
        switch (ch.nl) {
        case 1: assemble_grp_body<BD, 1>(A, ch, sp, sc, idx, G, Wh, Wl); break;
        case 2: assemble_grp_body<BD, 2>(A, ch, sp, sc, idx, G, Wh, Wl); break;
        case 3: assemble_grp_body<BD, 3>(A, ch, sp, sc, idx, G, Wh, Wl); break;
        default: assemble_grp_body<BD, 4>(A, ch, sp, sc, idx, G, Wh, Wl); break;
        }
    }
}

void launch_assemble_grp_df(cudaStream_t st, const OpView& A, const AsmChunk* chunks, int nchunks, const int* gpair,
                            const float4* gcoef, const float2* G, float* Wh, float* Wl)
{
    dim3 grid((unsigned)((A.n1 * A.bd + 127) / 128), (unsigned)std::min(nchunks, 65535));
    if (A.bd == 13) k_assemble_grp_df<13><<<grid, 128, 0, st>>>(A, chunks, nchunks, gpair, gcoef, G, Wh, Wl);
    else k_assemble_grp_df<0><<<grid, 128, 0, st>>>(A, chunks, nchunks, gpair, gcoef, G, Wh, Wl);
}

// u = psi + x, v = psi - x in double, each split into (re_hi, re_lo, im_hi, im_lo)
__global__ void k_split_uv(int64_t n, const double2* __restrict__ psi, const double2* __restrict__ x,
                           float4* __restrict__ u, float4* __restrict__ v)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 p = psi[i], q = x[i];
    float2 a = df_split(p.x + q.x), b = df_split(p.y + q.y), c = df_split(p.x - q.x), d = df_split(p.y - q.y);
    u[i] = make_float4(a.x, a.y, b.x, b.y);
    v[i] = make_float4(c.x, c.y, d.x, d.y);
}

// u = psi + x, v = psi - x (split) and psi rounded to FP32.  u and v are stored type-major within
// each channel, [channel][DKB type][radial slot] (n1 = slots per channel), so that each type's rows
// are 16 B apart: the owner pass copies a type's window as one contiguous range and its threads
// read consecutive rows without shared-memory bank conflicts.  psi32 keeps the state's order.
__global__ void k_split_uv3(int64_t n, int n1, const double2* __restrict__ psi, const double2* __restrict__ x,
                            float4* __restrict__ u, float4* __restrict__ v, float2* __restrict__ psi32)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 p = psi[i], q = x[i];
    // the sums exact in FP64 (4 additions), their splits and psi's hi words by integer operations
    float2 a = df_split_bits(p.x + q.x), b = df_split_bits(p.y + q.y), c = df_split_bits(p.x - q.x),
           d = df_split_bits(p.y - q.y);
    const int64_t ch = i / (2 * n1);
    const int rem = (int)(i - ch * 2 * n1), r = rem >> 1, t = rem & 1;
    const int64_t o = (ch * 2 + t) * n1 + r;
    u[o] = make_float4(a.x, a.y, b.x, b.y);
    v[o] = make_float4(c.x, c.y, d.x, d.y);
    psi32[i] = make_float2(df_split_bits(p.x).x, df_split_bits(p.y).x);
}

// Refinement residual r = A_- psi - A_+ x in double-float through one coupling product:
//   r = S (psi - x) - i tau H0 (psi + x) + (W - W^T)(psi + x)
// (A_-+ = S -+ i tau H0 +- (W - W^T) with W the stored upper-pair coupling, Eq. solPsi and
// Eq. fullH), from u = psi + x and v = psi - x.  Also ||b||^2 of b = A_- psi (the tolerance
// scale) from FP32 products of psi = (u + v)/2.  Output r in double; partials of ||r||^2, ||b||^2.
template <int BD>
__global__ void __launch_bounds__(128) k_residual_df(OpView A, const float2* __restrict__ S, const float2* __restrict__ Ht,
                                                     const float4* __restrict__ u, const float4* __restrict__ v,
                                                     const float* __restrict__ Wh, const float* __restrict__ Wl,
                                                     double2* __restrict__ r_out, double* part_r, double* part_b)
{
    const int bd = BD > 0 ? BD : A.bd;
    const int half = (bd - 1) / 2;
    const int n1 = A.n1;
    int ch = blockIdx.x;   // tile-major, as the operator apply
    int r = blockIdx.y * blockDim.x + threadIdx.x;
    double nr = 0, nbv = 0;
    if (r < n1) {
        const float4* ua = u + (int64_t)ch * 2 * n1;
        const float4* va = v + (int64_t)ch * 2 * n1;
        int ks = A.ch_kslot[ch];
        const float2* Sk = S + ((int64_t)ks * n1 + r) * bd * 4;
        const float2* Hk = Ht + ((int64_t)ks * n1 + r) * bd * 4;
        DfAcc yv[4];   // (row type 0 re, im, row type 1 re, im)
        for (int k = 0; k < 4; k++) df_zero(yv[k]);
        float bb[4] = {0.f, 0.f, 0.f, 0.f};   // b = A_- psi, FP32 (tolerance scale only)
#pragma unroll
        for (int d = 0; d < bd; d++) {
            int rr = r + d - half;
            if (rr < 0 || rr >= n1) continue;
            float4 u0 = ua[2 * rr], u1 = ua[2 * rr + 1], v0 = va[2 * rr], v1 = va[2 * rr + 1];
            float p0r = 0.5f * (u0.x + v0.x), p0i = 0.5f * (u0.z + v0.z);
            float p1r = 0.5f * (u1.x + v1.x), p1i = 0.5f * (u1.z + v1.z);
            for (int t = 0; t < 2; t++) {
                float2 s0 = Sk[d * 4 + 2 * t], s1 = Sk[d * 4 + 2 * t + 1];
                float2 h0 = Hk[d * 4 + 2 * t], h1 = Hk[d * 4 + 2 * t + 1];
                // re: S v_re + tau H u_im ;  im: S v_im - tau H u_re
                df_fma(yv[2 * t], s0.x, s0.y, v0.x, v0.y);
                df_fma(yv[2 * t], s1.x, s1.y, v1.x, v1.y);
                df_fma(yv[2 * t], h0.x, h0.y, u0.z, u0.w);
                df_fma(yv[2 * t], h1.x, h1.y, u1.z, u1.w);
                df_fma(yv[2 * t + 1], s0.x, s0.y, v0.z, v0.w);
                df_fma(yv[2 * t + 1], s1.x, s1.y, v1.z, v1.w);
                df_fma(yv[2 * t + 1], -h0.x, -h0.y, u0.x, u0.y);
                df_fma(yv[2 * t + 1], -h1.x, -h1.y, u1.x, u1.y);
                // b = (S - i tau H) psi
                bb[2 * t] += s0.x * p0r + s1.x * p1r + h0.x * p0i + h1.x * p1i;
                bb[2 * t + 1] += s0.x * p0i + s1.x * p1i - h0.x * p0r - h1.x * p1r;
            }
        }
        // coupling: + W u (this channel is the pair's lower one), - W^T u (upper one)
        for (int e = A.adj_start[ch]; e < A.adj_start[ch + 1]; e++) {
            int64_t p = A.adj_pair[e];
            const float4* ub = u + (int64_t)A.adj_nbr[e] * 2 * n1;
            const float4* vb = v + (int64_t)A.adj_nbr[e] * 2 * n1;
            const float* Whp = Wh + p * n1 * bd * 4;
            const float* Wlp = Wl + p * n1 * bd * 4;
            bool tr = A.adj_tr[e];
            float sg = tr ? -1.f : 1.f;
#pragma unroll
            for (int d = 0; d < bd; d++) {
                int rr = r + d - half;
                if (rr < 0 || rr >= n1) continue;
                float4 x0 = ub[2 * rr], x1 = ub[2 * rr + 1];
                float4 y0 = vb[2 * rr], y1 = vb[2 * rr + 1];
                int64_t o = tr ? ((int64_t)rr * bd + (2 * half - d)) * 4 : ((int64_t)r * bd + d) * 4;
                float4 wh = *reinterpret_cast<const float4*>(Whp + o);
                float4 wl = *reinterpret_cast<const float4*>(Wlp + o);
                // row t of the block applied: direct W[t][u] = (x, y; z, w), transposed W[u][t]
                float a00 = sg * wh.x, a01 = sg * (tr ? wh.z : wh.y), a10 = sg * (tr ? wh.y : wh.z), a11 = sg * wh.w;
                float l00 = sg * wl.x, l01 = sg * (tr ? wl.z : wl.y), l10 = sg * (tr ? wl.y : wl.z), l11 = sg * wl.w;
                df_fma(yv[0], a00, l00, x0.x, x0.y); df_fma(yv[0], a01, l01, x1.x, x1.y);
                df_fma(yv[1], a00, l00, x0.z, x0.w); df_fma(yv[1], a01, l01, x1.z, x1.w);
                df_fma(yv[2], a10, l10, x0.x, x0.y); df_fma(yv[2], a11, l11, x1.x, x1.y);
                df_fma(yv[3], a10, l10, x0.z, x0.w); df_fma(yv[3], a11, l11, x1.z, x1.w);
                float q0r = 0.5f * (x0.x + y0.x), q0i = 0.5f * (x0.z + y0.z);
                float q1r = 0.5f * (x1.x + y1.x), q1i = 0.5f * (x1.z + y1.z);
                bb[0] += a00 * q0r + a01 * q1r;
                bb[1] += a00 * q0i + a01 * q1i;
                bb[2] += a10 * q0r + a11 * q1r;
                bb[3] += a10 * q0i + a11 * q1i;
            }
        }
        int64_t o = (int64_t)ch * 2 * n1 + 2 * r;
        double2 y0 = make_double2(df_value(yv[0]), df_value(yv[1])), y1 = make_double2(df_value(yv[2]), df_value(yv[3]));
        r_out[o] = y0;
        r_out[o + 1] = y1;
        nr = y0.x * y0.x + y0.y * y0.y + y1.x * y1.x + y1.y * y1.y;
        for (int k = 0; k < 4; k++) nbv += (double)bb[k] * bb[k];
    }
    int64_t slot = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    block_reduce_store(make_double2(0, 0), nr, nullptr, part_r, slot);
    block_reduce_store(make_double2(0, 0), nbv, nullptr, part_b, slot);
}

void launch_residual_df(dim3 grid, cudaStream_t st, const OpView& A, const float2* S, const float2* Ht, const float4* u,
                        const float4* v, const float* Wh, const float* Wl, double2* r, double* pr, double* pb)
{
    if (A.bd == 13) k_residual_df<13><<<grid, 128, 0, st>>>(A, S, Ht, u, v, Wh, Wl, r, pr, pb);
    else k_residual_df<0><<<grid, 128, 0, st>>>(A, S, Ht, u, v, Wh, Wl, r, pr, pb);
}

// y = A_sign x in double-float (x split into float4 per complex); output in double:
// y <- bsub - y when bsub is given; partial ||y||^2 per block.  Diagonal blocks: S and tau H0 as
// float2 (hi, lo) per entry.
template <int BD>
__global__ void __launch_bounds__(128) k_apply_df(OpView A, const float2* __restrict__ S, const float2* __restrict__ Ht,
                                                  int sign, const float4* __restrict__ x, const float* __restrict__ Wh,
                                                  const float* __restrict__ Wl, double2* __restrict__ y,
                                                  const double2* __restrict__ bsub, double* part_nrm)
{
    const int bd = BD > 0 ? BD : A.bd;
    const int half = (bd - 1) / 2;
    const int n1 = A.n1;
    int ch = blockIdx.x;   // tile-major: see k_apply
    int r = blockIdx.y * blockDim.x + threadIdx.x;
    double nsum = 0;
    if (r < n1) {
        const float4* xa = x + (int64_t)ch * 2 * n1;
        int ks = A.ch_kslot[ch];
        const float2* Sk = S + ((int64_t)ks * n1 + r) * bd * 4;
        const float2* Hk = Ht + ((int64_t)ks * n1 + r) * bd * 4;
        float sg = (float)sign;
        // acc[0..3] = (y0 re, y0 im, y1 re, y1 im)
        DfAcc yv[4], dd[4], tt[4];
        for (int k = 0; k < 4; k++) { df_zero(yv[k]); df_zero(dd[k]); df_zero(tt[k]); }
#pragma unroll
        for (int d = 0; d < bd; d++) {
            int rr = r + d - half;
            if (rr < 0 || rr >= n1) continue;
            float4 x0 = xa[2 * rr], x1 = xa[2 * rr + 1];
            for (int t = 0; t < 2; t++) {
                float2 s0 = Sk[d * 4 + 2 * t], s1 = Sk[d * 4 + 2 * t + 1];
                float2 h0 = Hk[d * 4 + 2 * t], h1 = Hk[d * 4 + 2 * t + 1];
                // re += S x_re - sign tau H x_im ;  im += S x_im + sign tau H x_re
                df_fma(yv[2 * t], s0.x, s0.y, x0.x, x0.y);
                df_fma(yv[2 * t], s1.x, s1.y, x1.x, x1.y);
                df_fma(yv[2 * t], -sg * h0.x, -sg * h0.y, x0.z, x0.w);
                df_fma(yv[2 * t], -sg * h1.x, -sg * h1.y, x1.z, x1.w);
                df_fma(yv[2 * t + 1], s0.x, s0.y, x0.z, x0.w);
                df_fma(yv[2 * t + 1], s1.x, s1.y, x1.z, x1.w);
                df_fma(yv[2 * t + 1], sg * h0.x, sg * h0.y, x0.x, x0.y);
                df_fma(yv[2 * t + 1], sg * h1.x, sg * h1.y, x1.x, x1.y);
            }
        }
        for (int e = A.adj_start[ch]; e < A.adj_start[ch + 1]; e++) {
            int64_t p = A.adj_pair[e];
            const float4* xb = x + (int64_t)A.adj_nbr[e] * 2 * n1;
            const float* Whp = Wh + p * n1 * bd * 4;
            const float* Wlp = Wl + p * n1 * bd * 4;
            if (!A.adj_tr[e]) {
#pragma unroll
                for (int d = 0; d < bd; d++) {
                    int rr = r + d - half;
                    if (rr < 0 || rr >= n1) continue;
                    float4 x0 = xb[2 * rr], x1 = xb[2 * rr + 1];
                    float4 wh = *reinterpret_cast<const float4*>(Whp + ((int64_t)r * bd + d) * 4);
                    float4 wl = *reinterpret_cast<const float4*>(Wlp + ((int64_t)r * bd + d) * 4);
                    // W[t][u] = (w.x, w.y ; w.z, w.w)
                    df_fma(dd[0], wh.x, wl.x, x0.x, x0.y); df_fma(dd[0], wh.y, wl.y, x1.x, x1.y);
                    df_fma(dd[1], wh.x, wl.x, x0.z, x0.w); df_fma(dd[1], wh.y, wl.y, x1.z, x1.w);
                    df_fma(dd[2], wh.z, wl.z, x0.x, x0.y); df_fma(dd[2], wh.w, wl.w, x1.x, x1.y);
                    df_fma(dd[3], wh.z, wl.z, x0.z, x0.w); df_fma(dd[3], wh.w, wl.w, x1.z, x1.w);
                }
            } else {
#pragma unroll
                for (int d = 0; d < bd; d++) {
                    int rr = r + d - half;
                    if (rr < 0 || rr >= n1) continue;
                    float4 x0 = xb[2 * rr], x1 = xb[2 * rr + 1];
                    int64_t o = ((int64_t)rr * bd + (2 * half - d)) * 4;
                    float4 wh = *reinterpret_cast<const float4*>(Whp + o);
                    float4 wl = *reinterpret_cast<const float4*>(Wlp + o);
                    // (W^T)[t][u] = W[u][t]
                    df_fma(tt[0], wh.x, wl.x, x0.x, x0.y); df_fma(tt[0], wh.z, wl.z, x1.x, x1.y);
                    df_fma(tt[1], wh.x, wl.x, x0.z, x0.w); df_fma(tt[1], wh.z, wl.z, x1.z, x1.w);
                    df_fma(tt[2], wh.y, wl.y, x0.x, x0.y); df_fma(tt[2], wh.w, wl.w, x1.x, x1.y);
                    df_fma(tt[3], wh.y, wl.y, x0.z, x0.w); df_fma(tt[3], wh.w, wl.w, x1.z, x1.w);
                }
            }
        }
        double out[4];
        for (int k = 0; k < 4; k++) {
            df_add(yv[k], tt[k], sg);
            df_add(yv[k], dd[k], -sg);
            out[k] = df_value(yv[k]);
        }
        int64_t o = (int64_t)ch * 2 * n1 + 2 * r;
        double2 y0 = make_double2(out[0], out[1]), y1 = make_double2(out[2], out[3]);
        if (bsub) {
            double2 b0 = bsub[o], b1 = bsub[o + 1];
            y0 = make_double2(b0.x - y0.x, b0.y - y0.y);
            y1 = make_double2(b1.x - y1.x, b1.y - y1.y);
        }
        y[o] = y0;
        y[o + 1] = y1;
        nsum = y0.x * y0.x + y0.y * y0.y + y1.x * y1.x + y1.y * y1.y;
    }
    if (part_nrm) block_reduce_store(make_double2(0, 0), nsum, nullptr, part_nrm, (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
}

void launch_apply_df(dim3 grid, cudaStream_t st, const OpView& A, const float2* S, const float2* Ht, int sign,
                     const float4* x, const float* Wh, const float* Wl, double2* y, const double2* bsub, double* pn)
{
    if (A.bd == 13)
        k_apply_df<13><<<grid, 128, 0, st>>>(A, S, Ht, sign, x, Wh, Wl, y, bsub, pn);
    else
        k_apply_df<0><<<grid, 128, 0, st>>>(A, S, Ht, sign, x, Wh, Wl, y, bsub, pn);
}

}  // namespace dg
