// guess.cu -- the learned initial guess: a 4-layer network (32 -> 256 -> 256 -> 256 -> 4, tanh)
// that maps, per position (channel, radial slot), the last four states and the field to a
// correction of the extrapolated BiCGSTAB starting vector; its training (forward, backward, Adam)
// on the GPU.  Not part of the paper's method: it only moves the solver's starting point, and the
// solver's residual test still decides convergence.
//
// Per position p: the backward differences D_0..D_3 of psi_n .. psi_{n-3} at the slot (4 reals each:
// Re, Im of both DKB types), their rms m_k, s = m_3; features x = [D_k / m_k (16),
// clip(log10(m_j / m_3), -30, 30) / 10 (3), six field factors at t_{n+1}, kappa / 10, 2 mu / 20,
// zeros] (32); guess = 3 psi_n - 3 psi_{n-1} + psi_{n-2} + s * net(x).
// The weights are kept in FP32 for the optimiser and enter every product rounded to bfloat16;
// products accumulate in FP32.  Inference runs the three 256-wide layers on the tensor cores
// (bf16 mma.sync, FP32 accumulators); training runs FP32 tiled kernels on the same rounded weights.
// All reductions over samples (gradients, loss) are split in fixed chunks and summed in a fixed
// order, so training is reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dirac.h"
#include "device.h"
#include "internal.h"
#include "kernels.h"
#include "op.h"

namespace dg {

constexpr int GN_IN = 32, GN_H = 256, GN_OUT = 4;
// parameter layout (floats): W1 [32][256], b1, W2 [256][256], b2, W3 [256][256], b3, W4 [256][4], b4
constexpr int64_t GO_W1 = 0, GO_B1 = GO_W1 + GN_IN * GN_H, GO_W2 = GO_B1 + GN_H, GO_B2 = GO_W2 + GN_H * GN_H,
                  GO_W3 = GO_B2 + GN_H, GO_B3 = GO_W3 + GN_H * GN_H, GO_W4 = GO_B3 + GN_H,
                  GO_B4 = GO_W4 + GN_H * GN_OUT, GN_PARAMS = GO_B4 + GN_OUT;
constexpr int GCHUNK = 1024;   // samples per partial of a gradient reduction

}  // namespace dg

struct dirac_guess {
    int max_batch = 0;
    int64_t step = 0;               // Adam step count
    float* w = nullptr;             // FP32 master parameters
    float* wr = nullptr;            // the same with weights rounded to bf16 (biases unchanged)
    __nv_bfloat16* wb = nullptr;    // bf16 weights for the tensor-core forward (W1 padded, W4 padded to 8)
    __nv_bfloat16* wt = nullptr;    // the same, transposed and packed in the tcgen05 kernel's chunk layout
    int* err = nullptr;             // error word of the tcgen05 forward's bounded waits
    float *m = nullptr, *v = nullptr, *g = nullptr;
    float *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *out = nullptr;   // training activations
    float *d1 = nullptr, *d2 = nullptr, *dout = nullptr;                 // back-propagated errors
    float* part = nullptr;          // split-sample partial gradients
    double* lpart = nullptr;        // loss partials
    double* hloss = nullptr;        // pinned host loss
};

namespace dg {

// ------------------------------------------------------------------------------------------
// features and the guess
// ------------------------------------------------------------------------------------------
// field factors at t_next = t_start + (step + 1) dt (step >= 0), or at t_start itself (step < 0)
__global__ void k_guess_field(PulseView P, double t_start, int step, double dt, float* F)
{
    if (threadIdx.x || blockIdx.x) return;
    guess_field_at(P, step >= 0 ? next_time(t_start, step, dt) : t_start, F);
}

// one thread per position (channel, radial slot): backward differences D_0..D_3 of the four
// states, their rms m_k, x = [D_k / m_k, clip(log10(m_j / m_3)) / 10, field, kappa / 10, 2 mu / 20],
// s = m_3
// Features of one position (one thread), written through shared memory so that a warp stores
// whole 512-byte runs of X.  The backward differences need FP64 (they cancel to ~1e-6 of the
// states); everything after them runs in FP32 on a copy scaled by an exact power of two taken
// from the largest difference, so that neither the squares nor the normalisation under- or
// overflow (GB300's FP64 rate is 1/64 of FP32: a double sqrt, division and log10 per feature
// cost more than the rest of the guess).  The rms, the normalised differences and the log-ratios
// match the FP64 definition to FP32 rounding.
constexpr int GF_THREADS = 256;
__global__ void __launch_bounds__(GF_THREADS) k_guess_features(int nch, int n1, const int* __restrict__ kappa,
                                                               const int* __restrict__ two_mu,
                                                               const double2* __restrict__ p0,
                                                               const double2* __restrict__ p1,
                                                               const double2* __restrict__ p2,
                                                               const double2* __restrict__ p3,
                                                               const float* __restrict__ F, float* __restrict__ X,
                                                               float* __restrict__ S, const int* gate)
{
    __shared__ float xs[GF_THREADS * (GN_IN + 1)];   // +1: conflict-free column access
    if (gate && !*gate) return;   // uniform: the graph's step has too few past states
    const int64_t npos = (int64_t)nch * n1;
    const int64_t base = (int64_t)blockIdx.x * GF_THREADS;
    int64_t pos = base + threadIdx.x;
    float* xr = xs + threadIdx.x * (GN_IN + 1);
    if (pos < npos) {
        int ch = (int)(pos / n1);
        double D[4][4];
        for (int t = 0; t < 2; t++) {
            double2 a = p0[2 * pos + t], b = p1[2 * pos + t], c = p2[2 * pos + t], d = p3[2 * pos + t];
            double re[4] = {a.x, a.x - b.x, a.x - 2.0 * b.x + c.x, a.x - 3.0 * b.x + 3.0 * c.x - d.x};
            double im[4] = {a.y, a.y - b.y, a.y - 2.0 * b.y + c.y, a.y - 3.0 * b.y + 3.0 * c.y - d.y};
            for (int k = 0; k < 4; k++) {
                D[k][2 * t] = re[k];
                D[k][2 * t + 1] = im[k];
            }
        }
        float ms[4];   // rms of the scaled differences
        int ex[4];     // D[k] = Ds[k] 2^ex[k]
        for (int k = 0; k < 4; k++) {
            double amax = fmax(fmax(fabs(D[k][0]), fabs(D[k][1])), fmax(fabs(D[k][2]), fabs(D[k][3])));
            int e = 0;
            if (amax > 0) {
                // exponent of amax from its bit pattern (finite, nonzero): amax in [2^e, 2^(e+1))
                long long bits = __double_as_longlong(amax);
                int be = (int)((bits >> 52) & 0x7ff);
                e = be > 0 ? be - 1023 : -1022;   // subnormal differences: scale from 2^-1022
            }
            double sc = ldexp(1.0, -e);   // exact power of two
            float q = 0.f, v[4];
            for (int i = 0; i < 4; i++) {
                v[i] = (float)(D[k][i] * sc);
                q = fmaf(v[i], v[i], q);
            }
            ms[k] = sqrtf(0.25f * q);
            ex[k] = e;
            float inv = ms[k] > 0.f ? 1.f / ms[k] : 0.f;
            for (int i = 0; i < 4; i++) xr[4 * k + i] = v[i] * inv;
        }
        for (int j = 0; j < 3; j++) {
            float w = 0.f;
            if (ms[j] > 0.f && ms[3] > 0.f) {
                float lg = log10f(ms[j] / ms[3]) + (float)(ex[j] - ex[3]) * 0.30102999566398120f;
                w = fminf(30.f, fmaxf(-30.f, lg)) / 10.f;
            }
            xr[16 + j] = w;
        }
        for (int i = 0; i < 6; i++) xr[19 + i] = F[i];
        xr[25] = (float)kappa[ch] / 10.f;
        xr[26] = (float)two_mu[ch] / 20.f;
        for (int i = 27; i < GN_IN; i++) xr[i] = 0.f;
        S[pos] = ldexpf(ms[3], ex[3]);
    }
    __syncthreads();
    // block's rows of X, contiguous: element i of the block's run is row i / GN_IN, column i % GN_IN
    const int64_t nrows = min((int64_t)GF_THREADS, npos - base);
    float* Xb = X + base * GN_IN;
    for (int i = threadIdx.x; i < nrows * GN_IN; i += GF_THREADS) Xb[i] = xs[(i / GN_IN) * (GN_IN + 1) + i % GN_IN];
}

// target = (psi_{n+1} - x_ext) / s (zero where s = 0)
__global__ void k_guess_targets(int64_t npos, const double2* __restrict__ p0, const double2* __restrict__ p1,
                                const double2* __restrict__ p2, const double2* __restrict__ pn,
                                const float* __restrict__ S, float* __restrict__ T)
{
    int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= npos) return;
    float s = S[pos];
    double inv = s > 0 ? 1.0 / (double)s : 0.0;
    float o[4];
    for (int t = 0; t < 2; t++) {
        int64_t i = 2 * pos + t;
        double2 a = p0[i], b = p1[i], c = p2[i], y = pn[i];
        double xr = extrapolate(2, a.x, b.x, c.x), xi = extrapolate(2, a.y, b.y, c.y);
        o[2 * t] = (float)((y.x - xr) * inv);
        o[2 * t + 1] = (float)((y.y - xi) * inv);
    }
    *reinterpret_cast<float4*>(T + pos * 4) = make_float4(o[0], o[1], o[2], o[3]);
}

// x = x_ext + s * out
__global__ void k_guess_apply(int64_t npos, const double2* __restrict__ p0, const double2* __restrict__ p1,
                              const double2* __restrict__ p2, const float* __restrict__ S,
                              const float* __restrict__ out, double2* __restrict__ x, const int* gate)
{
    if (gate && !*gate) return;
    int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= npos) return;
    double s = S[pos];
    float4 o = *reinterpret_cast<const float4*>(out + pos * 4);
    double c[4] = {o.x, o.y, o.z, o.w};
    for (int t = 0; t < 2; t++) {
        int64_t i = 2 * pos + t;
        double2 a = p0[i], b = p1[i], d = p2[i];
        x[i] = make_double2(__dadd_rn(extrapolate(2, a.x, b.x, d.x), __dmul_rn(s, c[2 * t])),
                            __dadd_rn(extrapolate(2, a.y, b.y, d.y), __dmul_rn(s, c[2 * t + 1])));
    }
}

// ------------------------------------------------------------------------------------------
// FP32 tiled GEMM with epilogues (training path and the reference forward)
//   C[i][j] = epi( sum_k A[i][k] B'[k][j] ),  B' = B (K x N, row-major) or B^T (B is N x K)
//   epi: 0 = + bias, 1 = tanh(. + bias), 2 = . * (1 - G[i][j]^2) (back-propagation through tanh)
// 64 x 64 tile per block of 256 threads, 4 x 4 outputs per thread, K in chunks of 16.
// ------------------------------------------------------------------------------------------
template <bool TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A,
                                              const float* __restrict__ B, const float* __restrict__ bias,
                                              const float* __restrict__ G, float* __restrict__ C)
{
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            int ii = e / 16, kk = e % 16;
            int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < M && gk < K) ? A[(int64_t)gi * K + gk] : 0.f;
            int jj = e % 64, kb = e / 64;
            int gj = j0 + jj, gkb = k0 + kb;
            float bv = 0.f;
            if (gj < N && gkb < K) bv = TB ? B[(int64_t)gj * K + gkb] : B[(int64_t)gkb * N + gj];
            Bs[kb][jj] = bv;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; kk++) {
            float a[4], b[4];
            for (int q = 0; q < 4; q++) { a[q] = As[kk][ty * 4 + q]; b[q] = Bs[kk][tx * 4 + q]; }
            for (int p = 0; p < 4; p++)
                for (int q = 0; q < 4; q++) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
    for (int p = 0; p < 4; p++) {
        int gi = i0 + ty * 4 + p;
        if (gi >= M) continue;
        for (int q = 0; q < 4; q++) {
            int gj = j0 + tx * 4 + q;
            if (gj >= N) continue;
            float v = acc[p][q];
            if (EPI == 0) v += bias[gj];
            else if (EPI == 1) v = tanhf(v + bias[gj]);
            else { float gg = G[(int64_t)gi * N + gj]; v *= 1.f - gg * gg; }
            C[(int64_t)gi * N + gj] = v;
        }
    }
}

// partial weight gradient over one chunk of samples: P[chunk][k][j] = sum_{i in chunk} A[i][k] D[i][j]
// (A: M x K, D: M x N); a 64 x 64 (k, j) tile per block
__global__ void __launch_bounds__(256) k_gemm_tn_part(int M, int N, int K, const float* __restrict__ A,
                                                      const float* __restrict__ D, float* __restrict__ P)
{
    __shared__ float As[16][64 + 4];
    __shared__ float Ds[16][64 + 4];
    int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int k0 = blockIdx.y * 64, j0 = blockIdx.x * 64, chunk = blockIdx.z;
    int ib = chunk * GCHUNK, ie = min(M, ib + GCHUNK);
    float acc[4][4] = {};
    for (int i1 = ib; i1 < ie; i1 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            int ii = e / 64, cc = e % 64;
            int gi = i1 + ii;
            bool in = gi < ie;
            As[ii][cc] = (in && k0 + cc < K) ? A[(int64_t)gi * K + k0 + cc] : 0.f;
            Ds[ii][cc] = (in && j0 + cc < N) ? D[(int64_t)gi * N + j0 + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int ii = 0; ii < 16; ii++) {
            float a[4], d[4];
            for (int q = 0; q < 4; q++) { a[q] = As[ii][ty * 4 + q]; d[q] = Ds[ii][tx * 4 + q]; }
            for (int p = 0; p < 4; p++)
                for (int q = 0; q < 4; q++) acc[p][q] = fmaf(a[p], d[q], acc[p][q]);
        }
        __syncthreads();
    }
    for (int p = 0; p < 4; p++) {
        int gk = k0 + ty * 4 + p;
        if (gk >= K) continue;
        for (int q = 0; q < 4; q++) {
            int gj = j0 + tx * 4 + q;
            if (gj < N) P[((int64_t)chunk * K + gk) * N + gj] = acc[p][q];
        }
    }
}

// G[k][j] = sum over chunks (fixed order) of P[chunk][k][j]
__global__ void k_sum_chunks(int nchunk, int64_t KN, const float* __restrict__ P, float* __restrict__ G)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= KN) return;
    float s = 0.f;
    for (int c = 0; c < nchunk; c++) s += P[(int64_t)c * KN + e];
    G[e] = s;
}

// bias gradient: g[j] = sum_i D[i][j], chunked in the same fixed order
__global__ void k_colsum_part(int M, int N, const float* __restrict__ D, float* __restrict__ P)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x, chunk = blockIdx.y;
    if (j >= N) return;
    int ib = chunk * GCHUNK, ie = min(M, ib + GCHUNK);
    float s = 0.f;
    for (int i = ib; i < ie; i++) s += D[(int64_t)i * N + j];
    P[(int64_t)chunk * N + j] = s;
}

// dout = 2 (out - target) / B and per-chunk loss partials (double)
__global__ void k_loss_grad(int B, const float* __restrict__ out, const float* __restrict__ tgt,
                            float* __restrict__ dout, double* __restrict__ lpart)
{
    __shared__ double red[256];
    int chunk = blockIdx.x;
    int ib = chunk * GCHUNK, ie = min(B, ib + GCHUNK);
    double s = 0;
    for (int i = ib + threadIdx.x; i < ie; i += blockDim.x)
        for (int o = 0; o < GN_OUT; o++) {
            float d = out[(int64_t)i * GN_OUT + o] - tgt[(int64_t)i * GN_OUT + o];
            dout[(int64_t)i * GN_OUT + o] = 2.f * d / (float)B;
            s += (double)d * d;
        }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[chunk] = red[0];
}

__global__ void k_loss_sum(int n, const double* lpart, int B, double* out)
{
    if (threadIdx.x || blockIdx.x) return;
    double s = 0;
    for (int i = 0; i < n; i++) s += lpart[i];
    *out = s / B;
}

__device__ __forceinline__ bool is_weight(int64_t i)
{
    return (i >= GO_W1 && i < GO_B1) || (i >= GO_W2 && i < GO_B2) || (i >= GO_W3 && i < GO_B3) ||
           (i >= GO_W4 && i < GO_B4);
}

// rounded copies: wr = bf16(w) for weights (biases copied); wb = bf16 weights for the tensor
// cores, W1 and W4 stored as [32][256], [256][256], [256][256], [256][8] (W4 columns 4..7 zero)
__global__ void k_round_params(const float* __restrict__ w, float* __restrict__ wr, __nv_bfloat16* __restrict__ wb)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= GN_PARAMS) return;
    float v = w[i];
    if (is_weight(i)) {
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        wr[i] = __bfloat162float(b);
        int64_t o = -1;
        if (i < GO_B1) o = i;                                   // W1 [32][256]
        else if (i >= GO_W2 && i < GO_B2) o = GN_IN * GN_H + (i - GO_W2);
        else if (i >= GO_W3 && i < GO_B3) o = GN_IN * GN_H + GN_H * GN_H + (i - GO_W3);
        else if (i >= GO_W4 && i < GO_B4) {
            int64_t q = i - GO_W4;
            o = GN_IN * GN_H + 2 * GN_H * GN_H + (q / GN_OUT) * 8 + (q % GN_OUT);
        }
        wb[o] = b;
    } else {
        wr[i] = v;
    }
}

__global__ void k_adam(int64_t n, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------------------------------------
// Tensor-core forward: 64 positions per block (8 warps, each a 32-row x 64-column tile of every
// layer), bf16 mma.sync m16n8k16 with FP32 accumulators.  Activations stay in shared memory as
// bf16 (two 64 x 256 buffers); the 256 x 256 weights stream through shared memory in 32-row
// chunks, double buffered, once per layer; two blocks fit on an SM.
// ------------------------------------------------------------------------------------------
constexpr int FT_M = 64;                  // positions per block (two blocks per SM)
constexpr int FT_WM = 2, FT_WN = 4;       // warps along rows and along the 256 columns
constexpr int FT_THREADS = 32 * FT_WM * FT_WN;
constexpr int FT_MB = FT_M / FT_WM / 16;  // 16-row blocks per warp
constexpr int FT_JP = GN_H / FT_WN / 16;  // 16-column pairs of 8-column tiles per warp
constexpr int FT_KC = 32;                 // weight rows per chunk
constexpr int FT_AST = GN_H + 8;          // activation row stride (bf16), padded against bank conflicts
constexpr int FT_WST = GN_H + 8;          // weight chunk row stride (bf16)

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Fragments come from shared memory through ldmatrix (A: 16 x 16 activation tiles; B: the weight
// chunk [k][n] read transposed, two 8-column tiles at a time); weight chunks arrive by cp.async one
// chunk ahead of the chunk being multiplied.
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t* r, const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void cpa16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// FT_KC weight rows [k0, k0 + FT_KC) of a 256-wide bf16 matrix into a chunk buffer, asynchronously
__device__ __forceinline__ void ft_load_chunk_async(__nv_bfloat16* dst, const __nv_bfloat16* W, int k0)
{
    for (int e = threadIdx.x; e < FT_KC * GN_H / 8; e += blockDim.x) {
        int r = e / (GN_H / 8), c8 = e % (GN_H / 8);
        cpa16(dst + r * FT_WST + c8 * 8, W + (int64_t)(k0 + r) * GN_H + c8 * 8);
    }
    cpa_commit();
}

// hardware tanh (one MUFU instruction): relative error about 2^-11, below the bfloat16 rounding the
// activations get next; the FP32 kernels (training, reference forward) keep tanhf
__device__ __forceinline__ float tanh_hw(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(FT_THREADS) k_guess_forward_tc(int64_t M, const float* __restrict__ X,
                                                          const __nv_bfloat16* __restrict__ wb,
                                                          const float* __restrict__ wr, float* __restrict__ out,
                                                          const int* gate)
{
    if (gate && !*gate) return;
    extern __shared__ __align__(16) unsigned char ft_smem[];
    __nv_bfloat16* actA = reinterpret_cast<__nv_bfloat16*>(ft_smem);
    __nv_bfloat16* actB = actA + FT_M * FT_AST;
    __nv_bfloat16* wch = actB + FT_M * FT_AST;   // [2][FT_KC][FT_WST]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tq = lane & 3;       // mma fragment coordinates
    const int mi = lane >> 3, r8 = lane & 7;      // ldmatrix: matrix and row this lane addresses
    const int64_t m0 = (int64_t)blockIdx.x * FT_M;
    const __nv_bfloat16* W1 = wb;
    const __nv_bfloat16* W2 = wb + GN_IN * GN_H;
    const __nv_bfloat16* W3 = W2 + GN_H * GN_H;
    const __nv_bfloat16* W4 = W3 + GN_H * GN_H;   // [256][8]
    const float* b1 = wr + GO_B1;
    const float* b2 = wr + GO_B2;
    const float* b3 = wr + GO_B3;
    const float* b4 = wr + GO_B4;
    ft_load_chunk_async(wch, W1, 0);   // W1 is one chunk (32 rows)
    // stage X (bf16) into actB columns 0..31
    for (int e = threadIdx.x; e < FT_M * GN_IN; e += blockDim.x) {
        int r = e / GN_IN, c = e % GN_IN;
        int64_t gm = m0 + r;
        float v = gm < M ? X[gm * GN_IN + c] : 0.f;
        actB[r * FT_AST + c] = __float2bfloat16_rn(v);
    }
    cpa_wait0();
    __syncthreads();
    const int rw = warp * 16;   // the warp's rows in layer 4
    // A fragments of rows rw .. rw + 15, columns kk .. kk + 15 (layer 4)
    auto load_a = [&](const __nv_bfloat16* act, int kk, uint32_t* a) {
        ldsm_x4(a, act + (rw + (mi & 1) * 8 + r8) * FT_AST + kk + (mi >> 1) * 8);
    };
    // layers 1-3: FT_WM x FT_WN warps tile the FT_M-row x 256-column output (32 x 64 per warp), so
    // each B fragment feeds FT_MB row blocks and each A fragment FT_JP column pairs, and every
    // weight chunk is streamed once per layer
    const int wm = warp / FT_WN, wn = warp % FT_WN;
    const int rwm = wm * FT_MB * 16, cwn = wn * FT_JP * 16;
    auto mma_step = [&](const __nv_bfloat16* act, int ka, const __nv_bfloat16* w, int kw,
                        float (&acc)[FT_MB][2 * FT_JP][4]) {
        uint32_t a[FT_MB][4];
#pragma unroll
        for (int mb = 0; mb < FT_MB; mb++)
            ldsm_x4(a[mb], act + (rwm + mb * 16 + (mi & 1) * 8 + r8) * FT_AST + ka + (mi >> 1) * 8);
#pragma unroll
        for (int jp = 0; jp < FT_JP; jp++) {
            uint32_t bf[4];
            ldsm_x4_trans(bf, w + (kw + (mi & 1) * 8 + r8) * FT_WST + cwn + jp * 16 + (mi >> 1) * 8);
#pragma unroll
            for (int mb = 0; mb < FT_MB; mb++) {
                mma_bf16(acc[mb][2 * jp], a[mb], bf);
                mma_bf16(acc[mb][2 * jp + 1], a[mb], bf + 2);
            }
        }
    };
    // tanh(acc + bias) as bf16 into the output activations (the thread's rows and columns)
    auto epilogue = [&](float (&acc)[FT_MB][2 * FT_JP][4], const float* bias, __nv_bfloat16* outb) {
#pragma unroll
        for (int mb = 0; mb < FT_MB; mb++)
#pragma unroll
            for (int j = 0; j < 2 * FT_JP; j++) {
                int c = cwn + j * 8 + 2 * tq;
                float bb0 = bias[c], bb1 = bias[c + 1];
                int r = rwm + mb * 16 + g;
                *reinterpret_cast<uint32_t*>(outb + r * FT_AST + c) =
                    pack_bf16(tanh_hw(acc[mb][j][0] + bb0), tanh_hw(acc[mb][j][1] + bb1));
                *reinterpret_cast<uint32_t*>(outb + (r + 8) * FT_AST + c) =
                    pack_bf16(tanh_hw(acc[mb][j][2] + bb0), tanh_hw(acc[mb][j][3] + bb1));
            }
    };
    // layer 1: actB[:, 0:32] x W1 -> tanh -> actA
    {
        float acc[FT_MB][2 * FT_JP][4];
        for (int mb = 0; mb < FT_MB; mb++)
            for (int j = 0; j < 2 * FT_JP; j++)
                for (int q = 0; q < 4; q++) acc[mb][j][q] = 0.f;
        for (int kk = 0; kk < GN_IN; kk += 16) mma_step(actB, kk, wch, kk, acc);
        epilogue(acc, b1, actA);
    }
    __syncthreads();
    // layers 2 and 3: in -> out, weights streamed in FT_KC-row chunks, one chunk ahead
    constexpr int NCH = GN_H / FT_KC;
    for (int layer = 0; layer < 2; layer++) {
        const __nv_bfloat16* W = layer == 0 ? W2 : W3;
        const float* bias = layer == 0 ? b2 : b3;
        __nv_bfloat16* in = layer == 0 ? actA : actB;
        __nv_bfloat16* outb = layer == 0 ? actB : actA;
        {
            float acc[FT_MB][2 * FT_JP][4];
            for (int mb = 0; mb < FT_MB; mb++)
                for (int j = 0; j < 2 * FT_JP; j++)
                    for (int q = 0; q < 4; q++) acc[mb][j][q] = 0.f;
            ft_load_chunk_async(wch, W, 0);
            for (int c = 0; c < NCH; c++) {
                if (c + 1 < NCH) {
                    ft_load_chunk_async(wch + ((c + 1) & 1) * FT_KC * FT_WST, W, (c + 1) * FT_KC);
                    cpa_wait1();
                } else {
                    cpa_wait0();
                }
                __syncthreads();
                const __nv_bfloat16* cur = wch + (c & 1) * FT_KC * FT_WST;
                for (int kk = 0; kk < FT_KC; kk += 16) mma_step(in, c * FT_KC + kk, cur, kk, acc);
                __syncthreads();   // buffer (c & 1) is refilled two chunks later
            }
            epilogue(acc, bias, outb);
        }
        __syncthreads();
    }
    // layer 4: actA x W4 (256 x 8, columns 4..7 zero) -> out (FP32), warps 0..7 (16 rows each)
    if (warp < FT_M / 16) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int kk = 0; kk < GN_H; kk += 16) {
            uint32_t a[4], b[2];
            load_a(actA, kk, a);
            __nv_bfloat162 p0, p1;
            p0.x = W4[(kk + 2 * tq) * 8 + g];
            p0.y = W4[(kk + 2 * tq + 1) * 8 + g];
            p1.x = W4[(kk + 2 * tq + 8) * 8 + g];
            p1.y = W4[(kk + 2 * tq + 9) * 8 + g];
            b[0] = *reinterpret_cast<uint32_t*>(&p0);
            b[1] = *reinterpret_cast<uint32_t*>(&p1);
            mma_bf16(acc, a, b);
        }
        // acc[0..1]: row rw+g, cols 2tq, 2tq+1; acc[2..3]: row rw+g+8
        int c = 2 * tq;
        if (c < GN_OUT) {
            int64_t ra = m0 + rw + g, rb = m0 + rw + g + 8;
            if (ra < M) { out[ra * GN_OUT + c] = acc[0] + b4[c]; out[ra * GN_OUT + c + 1] = acc[1] + b4[c + 1]; }
            if (rb < M) { out[rb * GN_OUT + c] = acc[2] + b4[c]; out[rb * GN_OUT + c + 1] = acc[3] + b4[c + 1]; }
        }
    }
}

size_t guess_forward_tc_smem() { return sizeof(__nv_bfloat16) * (2 * FT_M * FT_AST + 2 * FT_KC * FT_WST); }

}  // namespace dg

using namespace dg;

namespace {

dirac_status gcheck(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return DIRAC_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? DIRAC_E_NOMEM : DIRAC_E_CUDA;
}

#define GTRY(call, what)                                  \
    do {                                                  \
        dirac_status s_ = gcheck((call), what);           \
        if (s_) return s_;                                \
    } while (0)

int nchunks(int B) { return (B + GCHUNK - 1) / GCHUNK; }

// forward through the FP32 kernels, keeping the activations (training and the reference path)
void fwd32(dirac_guess* g, const float* X, int B, cudaStream_t st)
{
    dim3 b(256);
    const float* wr = g->wr;
    k_gemm<false, 1><<<dim3(GN_H / 64, (B + 63) / 64), b, 0, st>>>(B, GN_H, GN_IN, X, wr + GO_W1, wr + GO_B1, nullptr, g->a1);
    k_gemm<false, 1><<<dim3(GN_H / 64, (B + 63) / 64), b, 0, st>>>(B, GN_H, GN_H, g->a1, wr + GO_W2, wr + GO_B2, nullptr, g->a2);
    k_gemm<false, 1><<<dim3(GN_H / 64, (B + 63) / 64), b, 0, st>>>(B, GN_H, GN_H, g->a2, wr + GO_W3, wr + GO_B3, nullptr, g->a3);
    k_gemm<false, 0><<<dim3(1, (B + 63) / 64), b, 0, st>>>(B, GN_OUT, GN_H, g->a3, wr + GO_W4, wr + GO_B4, nullptr, g->out);
}

// loss and gradient into g->g (all parameters), loss partials into g->lpart
void bwd32(dirac_guess* g, const float* X, const float* T, int B, cudaStream_t st)
{
    int nc = nchunks(B);
    dim3 b(256);
    const float* wr = g->wr;
    float* P = g->part;
    k_loss_grad<<<nc, 256, 0, st>>>(B, g->out, T, g->dout, g->lpart);
    // layer 4
    k_gemm_tn_part<<<dim3(1, GN_H / 64, nc), b, 0, st>>>(B, GN_OUT, GN_H, g->a3, g->dout, P);
    k_sum_chunks<<<(GN_H * GN_OUT + 255) / 256, 256, 0, st>>>(nc, GN_H * GN_OUT, P, g->g + GO_W4);
    k_colsum_part<<<dim3(1, nc), 256, 0, st>>>(B, GN_OUT, g->dout, P);
    k_sum_chunks<<<1, 256, 0, st>>>(nc, GN_OUT, P, g->g + GO_B4);
    // d3 = (dout W4^T) (1 - a3^2) into d1 (scratch), then layer 3
    k_gemm<true, 2><<<dim3(GN_H / 64, (B + 63) / 64), b, 0, st>>>(B, GN_H, GN_OUT, g->dout, wr + GO_W4, nullptr, g->a3, g->d1);
    k_gemm_tn_part<<<dim3(GN_H / 64, GN_H / 64, nc), b, 0, st>>>(B, GN_H, GN_H, g->a2, g->d1, P);
    k_sum_chunks<<<(GN_H * GN_H + 255) / 256, 256, 0, st>>>(nc, GN_H * GN_H, P, g->g + GO_W3);
    k_colsum_part<<<dim3(1, nc), 256, 0, st>>>(B, GN_H, g->d1, P);
    k_sum_chunks<<<1, 256, 0, st>>>(nc, GN_H, P, g->g + GO_B3);
    // d2 = (d3 W3^T) (1 - a2^2), layer 2
    k_gemm<true, 2><<<dim3(GN_H / 64, (B + 63) / 64), b, 0, st>>>(B, GN_H, GN_H, g->d1, wr + GO_W3, nullptr, g->a2, g->d2);
    k_gemm_tn_part<<<dim3(GN_H / 64, GN_H / 64, nc), b, 0, st>>>(B, GN_H, GN_H, g->a1, g->d2, P);
    k_sum_chunks<<<(GN_H * GN_H + 255) / 256, 256, 0, st>>>(nc, GN_H * GN_H, P, g->g + GO_W2);
    k_colsum_part<<<dim3(1, nc), 256, 0, st>>>(B, GN_H, g->d2, P);
    k_sum_chunks<<<1, 256, 0, st>>>(nc, GN_H, P, g->g + GO_B2);
    // d1 = (d2 W2^T) (1 - a1^2), layer 1
    k_gemm<true, 2><<<dim3(GN_H / 64, (B + 63) / 64), b, 0, st>>>(B, GN_H, GN_H, g->d2, wr + GO_W2, nullptr, g->a1, g->d1);
    k_gemm_tn_part<<<dim3(GN_H / 64, 1, nc), b, 0, st>>>(B, GN_H, GN_IN, X, g->d1, P);
    k_sum_chunks<<<(GN_IN * GN_H + 255) / 256, 256, 0, st>>>(nc, GN_IN * GN_H, P, g->g + GO_W1);
    k_colsum_part<<<dim3(1, nc), 256, 0, st>>>(B, GN_H, g->d1, P);
    k_sum_chunks<<<1, 256, 0, st>>>(nc, GN_H, P, g->g + GO_B1);
    k_loss_sum<<<1, 1, 0, st>>>(nc, g->lpart, B, g->lpart + nc);
}

}  // namespace

extern "C" int64_t dirac_guess_param_count(void) { return GN_PARAMS; }

extern "C" dirac_status dirac_guess_create(int max_batch, dirac_guess** out)
{
    if (!out || max_batch <= 0) { set_error("dirac_guess_create: bad argument"); return DIRAC_E_ARG; }
    *out = nullptr;
    dirac_guess* g = new dirac_guess();
    g->max_batch = max_batch;
    int nc = nchunks(max_batch);
    size_t act = (size_t)max_batch * GN_H;
    cudaError_t e = cudaSuccess;
    auto al = [&](auto** p, size_t count) {
        if (e == cudaSuccess) e = cudaMalloc((void**)p, sizeof(**p) * std::max<size_t>(count, 1));
    };
    al(&g->w, GN_PARAMS); al(&g->wr, GN_PARAMS); al(&g->m, GN_PARAMS); al(&g->v, GN_PARAMS); al(&g->g, GN_PARAMS);
    al(&g->wb, (size_t)GN_IN * GN_H + 2 * GN_H * GN_H + GN_H * 8);
    al(&g->wt, (size_t)guess_tc05_packed());
    al(&g->err, 1);
    al(&g->a1, act); al(&g->a2, act); al(&g->a3, act); al(&g->d1, act); al(&g->d2, act);
    al(&g->out, (size_t)max_batch * GN_OUT); al(&g->dout, (size_t)max_batch * GN_OUT);
    al(&g->part, (size_t)nc * GN_H * GN_H); al(&g->lpart, (size_t)nc + 1);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&g->hloss, sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(g->wb, 0, sizeof(__nv_bfloat16) * ((size_t)GN_IN * GN_H + 2 * GN_H * GN_H + GN_H * 8));
    if (e == cudaSuccess) e = cudaMemset(g->wt, 0, sizeof(__nv_bfloat16) * (size_t)guess_tc05_packed());
    if (e == cudaSuccess) e = cudaMemset(g->err, 0, sizeof(int));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_guess_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)guess_forward_tc_smem());
    if (e == cudaSuccess) e = guess_tc05_prepare();
    if (e != cudaSuccess) {
        set_error(std::string("dirac_guess_create: ") + cudaGetErrorString(e));
        dirac_guess_free(g);
        return e == cudaErrorMemoryAllocation ? DIRAC_E_NOMEM : DIRAC_E_CUDA;
    }
    *out = g;
    return DIRAC_OK;
}

extern "C" void dirac_guess_free(dirac_guess* g)
{
    if (!g) return;
    cudaDeviceSynchronize();
    for (void* p : {(void*)g->w, (void*)g->wr, (void*)g->wb, (void*)g->wt, (void*)g->err, (void*)g->m, (void*)g->v, (void*)g->g, (void*)g->a1,
                    (void*)g->a2, (void*)g->a3, (void*)g->out, (void*)g->d1, (void*)g->d2, (void*)g->dout,
                    (void*)g->part, (void*)g->lpart})
        cudaFree(p);
    cudaFreeHost(g->hloss);
    delete g;
}

extern "C" dirac_status dirac_guess_set_params(dirac_guess* g, const float* host, int64_t count)
{
    if (!g || !host || count != GN_PARAMS) { set_error("dirac_guess_set_params: bad argument"); return DIRAC_E_ARG; }
    GTRY(cudaMemcpy(g->w, host, sizeof(float) * GN_PARAMS, cudaMemcpyHostToDevice), "dirac_guess_set_params");
    GTRY(cudaMemset(g->m, 0, sizeof(float) * GN_PARAMS), "dirac_guess_set_params");
    GTRY(cudaMemset(g->v, 0, sizeof(float) * GN_PARAMS), "dirac_guess_set_params");
    g->step = 0;
    k_round_params<<<(GN_PARAMS + 255) / 256, 256>>>(g->w, g->wr, g->wb);
    launch_pack_tc05(nullptr, g->wb, g->wt);
    GTRY(cudaDeviceSynchronize(), "dirac_guess_set_params");
    return DIRAC_OK;
}

extern "C" dirac_status dirac_guess_get_params(dirac_guess* g, float* host, int64_t count)
{
    if (!g || !host || count != GN_PARAMS) { set_error("dirac_guess_get_params: bad argument"); return DIRAC_E_ARG; }
    GTRY(cudaDeviceSynchronize(), "dirac_guess_get_params");
    GTRY(cudaMemcpy(host, g->w, sizeof(float) * GN_PARAMS, cudaMemcpyDeviceToHost), "dirac_guess_get_params");
    return DIRAC_OK;
}

extern "C" dirac_status dirac_guess_features(dirac_op* op, const void* const* states, double t_next, float* x_dev,
                                             float* s_dev)
{
    if (!op || !states || !x_dev || !s_dev) { set_error("dirac_guess_features: bad argument"); return DIRAC_E_ARG; }
    for (int k = 0; k < 4; k++)
        if (!states[k]) { set_error("dirac_guess_features: NULL state"); return DIRAC_E_ARG; }
    int64_t npos = (int64_t)op->ov.nch * op->ov.n1;
    dirac_status fe = guess_buffers(op);
    if (fe) return fe;
    k_guess_field<<<1, 1, 0, op->st>>>(op->pv, t_next, -1, 0.0, op->gfield);
    k_guess_features<<<(unsigned)((npos + GF_THREADS - 1) / GF_THREADS), GF_THREADS, 0, op->st>>>(
        op->ov.nch, op->ov.n1, op->ov.ch_kappa, op->ch_two_mu, (const double2*)states[0], (const double2*)states[1],
        (const double2*)states[2], (const double2*)states[3], op->gfield, x_dev, s_dev, nullptr);
    op->launches += 2;
    return check_launch("dirac_guess_features");
}

extern "C" dirac_status dirac_guess_targets(dirac_op* op, const void* const* states, const void* psi_next,
                                            const float* s_dev, float* t_dev)
{
    if (!op || !states || !psi_next || !s_dev || !t_dev) { set_error("dirac_guess_targets: bad argument"); return DIRAC_E_ARG; }
    for (int k = 0; k < 3; k++)
        if (!states[k]) { set_error("dirac_guess_targets: NULL state"); return DIRAC_E_ARG; }
    int64_t npos = (int64_t)op->ov.nch * op->ov.n1;
    k_guess_targets<<<(unsigned)((npos + 255) / 256), 256, 0, op->st>>>(npos, (const double2*)states[0],
                                                                       (const double2*)states[1],
                                                                       (const double2*)states[2],
                                                                       (const double2*)psi_next, s_dev, t_dev);
    op->launches++;
    return check_launch("dirac_guess_targets");
}

extern "C" dirac_status dirac_guess_forward(dirac_guess* g, const float* x_dev, int64_t M, float* out_dev,
                                            int tensor_cores, void* stream)
{
    if (!g || !x_dev || !out_dev || M < 0 || tensor_cores < 0 || tensor_cores > 2) {
        set_error("dirac_guess_forward: bad argument");
        return DIRAC_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (M == 0) return DIRAC_OK;
    if (tensor_cores == 1) {
        launch_guess_forward_tc05(st, M, x_dev, g->wt, g->wr + GO_B1, g->wr + GO_B2, g->wr + GO_B3, g->wr + GO_B4,
                                  out_dev, nullptr, g->err);
        dirac_status e = check_launch("dirac_guess_forward");
        if (e) return e;
        int h = 0;
        GTRY(cudaMemcpyAsync(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost, st), "dirac_guess_forward");
        GTRY(cudaStreamSynchronize(st), "dirac_guess_forward");
        if (h) {
            GTRY(cudaMemsetAsync(g->err, 0, sizeof(int), st), "dirac_guess_forward");
            set_error("dirac_guess_forward: a bounded wait of the tcgen05 forward ran out of time (results invalid)");
            return DIRAC_E_CUDA;
        }
        return DIRAC_OK;
    }
    if (tensor_cores == 2) {
        k_guess_forward_tc<<<(unsigned)((M + FT_M - 1) / FT_M), FT_THREADS, guess_forward_tc_smem(), st>>>(
            M, x_dev, g->wb, g->wr, out_dev, nullptr);
        return check_launch("dirac_guess_forward");
    }
    // FP32 path in batches of max_batch samples (activations live in the training workspace)
    for (int64_t b0 = 0; b0 < M; b0 += g->max_batch) {
        int B = (int)std::min<int64_t>(g->max_batch, M - b0);
        fwd32(g, x_dev + b0 * GN_IN, B, st);
        GTRY(cudaMemcpyAsync(out_dev + b0 * GN_OUT, g->out, sizeof(float) * B * GN_OUT, cudaMemcpyDeviceToDevice, st),
             "dirac_guess_forward");
    }
    return check_launch("dirac_guess_forward");
}

extern "C" dirac_status dirac_guess_loss_grad(dirac_guess* g, const float* x_dev, const float* t_dev, int B,
                                              double* loss, float* grad_host, void* stream)
{
    if (!g || !x_dev || !t_dev || B <= 0 || B > g->max_batch) {
        set_error("dirac_guess_loss_grad: bad argument (0 < B <= max_batch)");
        return DIRAC_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    fwd32(g, x_dev, B, st);
    bwd32(g, x_dev, t_dev, B, st);
    dirac_status e = check_launch("dirac_guess_loss_grad");
    if (e) return e;
    GTRY(cudaMemcpyAsync(g->hloss, g->lpart + nchunks(B), sizeof(double), cudaMemcpyDeviceToHost, st),
         "dirac_guess_loss_grad");
    if (grad_host)
        GTRY(cudaMemcpyAsync(grad_host, g->g, sizeof(float) * GN_PARAMS, cudaMemcpyDeviceToHost, st),
             "dirac_guess_loss_grad");
    GTRY(cudaStreamSynchronize(st), "dirac_guess_loss_grad");
    if (loss) *loss = *g->hloss;
    return DIRAC_OK;
}

extern "C" dirac_status dirac_guess_train_step(dirac_guess* g, const float* x_dev, const float* t_dev, int B, double lr,
                                               double* loss, void* stream)
{
    if (!g || !x_dev || !t_dev || B <= 0 || B > g->max_batch || !(lr > 0)) {
        set_error("dirac_guess_train_step: bad argument (0 < B <= max_batch, lr > 0)");
        return DIRAC_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    fwd32(g, x_dev, B, st);
    bwd32(g, x_dev, t_dev, B, st);
    g->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = (float)(1.0 - std::pow(0.9, (double)g->step)), c2 = (float)(1.0 - std::pow(0.999, (double)g->step));
    k_adam<<<(GN_PARAMS + 255) / 256, 256, 0, st>>>(GN_PARAMS, g->w, g->m, g->v, g->g, (float)lr, b1, b2, 1e-8f, c1, c2);
    k_round_params<<<(GN_PARAMS + 255) / 256, 256, 0, st>>>(g->w, g->wr, g->wb);
    launch_pack_tc05(st, g->wb, g->wt);
    dirac_status e = check_launch("dirac_guess_train_step");
    if (e) return e;
    if (loss) {
        GTRY(cudaMemcpyAsync(g->hloss, g->lpart + nchunks(B), sizeof(double), cudaMemcpyDeviceToHost, st),
             "dirac_guess_train_step");
        GTRY(cudaStreamSynchronize(st), "dirac_guess_train_step");
        *loss = *g->hloss;
    }
    return DIRAC_OK;
}

// the learned guess inside a step: x = x_ext + s net(features), states psi_n, h1, h2, h3, the field
// at t_start + (step + 1) dt; with a gate (device flag) every kernel returns at once when it is 0
namespace dg {
dirac_status guess_buffers(dirac_op* op)
{
    if (op->gfield) return DIRAC_OK;
    GTRY(cudaMalloc(&op->gfield, sizeof(float) * 8), "learned guess");
    op->allocs.push_back(op->gfield);
    GTRY(cudaMalloc(&op->ggate, sizeof(int) * 4), "learned guess");
    op->allocs.push_back(op->ggate);
    return DIRAC_OK;
}

dirac_status guess_into(dirac_op* op, const double2* p0, const double2* h1, const double2* h2, const double2* h3,
                        double t_start, int step, double2* x, const int* gate, cudaStream_t st,
                        const float* field)
{
    dirac_guess* g = op->net;
    int64_t npos = (int64_t)op->ov.nch * op->ov.n1;
    unsigned nb = (unsigned)((npos + 255) / 256);
    if (!field) {
        k_guess_field<<<1, 1, 0, st>>>(op->pv, t_start, step, op->opts.dt, op->gfield);
        field = op->gfield;
        op->launches++;
    }
    k_guess_features<<<(unsigned)((npos + GF_THREADS - 1) / GF_THREADS), GF_THREADS, 0, st>>>(
        op->ov.nch, op->ov.n1, op->ov.ch_kappa, op->ch_two_mu, p0, h1, h2, h3, field, op->gx, op->gs, gate);
    launch_guess_forward_tc05(st, npos, op->gx, g->wt, g->wr + GO_B1, g->wr + GO_B2, g->wr + GO_B3, g->wr + GO_B4,
                              op->gout, gate, op->dev_err);
    k_guess_apply<<<nb, 256, 0, st>>>(npos, p0, h1, h2, op->gs, op->gout, x, gate);
    op->launches += 3;
    return check_launch("learned guess");
}
}  // namespace dg

extern "C" dirac_status dirac_op_set_guess(dirac_op* op, dirac_guess* net)
{
    if (!op) { set_error("dirac_op_set_guess: bad argument"); return DIRAC_E_ARG; }
    op->net = net;
    if (net && !op->gx) {
        int64_t npos = (int64_t)op->ov.nch * op->ov.n1;
        GTRY(cudaMalloc(&op->gx, sizeof(float) * npos * GN_IN), "dirac_op_set_guess");
        op->allocs.push_back(op->gx);
        GTRY(cudaMalloc(&op->gs, sizeof(float) * npos), "dirac_op_set_guess");
        op->allocs.push_back(op->gs);
        GTRY(cudaMalloc(&op->gout, sizeof(float) * npos * GN_OUT), "dirac_op_set_guess");
        op->allocs.push_back(op->gout);
        dirac_status e = guess_buffers(op);
        if (e) return e;
    }
    op->config_gen++;   // captured graphs take the network into account
    return DIRAC_OK;
}
