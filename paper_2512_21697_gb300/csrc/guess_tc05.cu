// guess_tc05.cu -- forward pass of the learned initial-guess network (32 -> 256 -> 256 -> 256 -> 4,
// tanh; bf16 weights and activations, FP32 accumulation) on the fifth-generation tensor cores:
// tcgen05.mma with the accumulators in tensor memory (TMEM).
//
// Block = 128 positions = one MMA tile (M = 128), 4 warps.  The tile's activations live in shared
// memory as bf16 in the K-major, no-swizzle operand layout of the MMA (8 x 8 core matrices of 128 B,
// row-group major: element (r, k) at (r / 8) * 4096 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
// bytes, so core matrices adjacent in K are 128 B apart and adjacent 8-row groups 4096 B).  The
// transposed weights are packed once per parameter update into the same layout, in 16 KB chunks of
// 32 K-rows x 256 outputs (W1: 1 chunk, W2 and W3: 8 each, W4: one 8 KB chunk of 256 K x 16
// outputs, columns 4..15 zero), so a chunk is one contiguous bulk copy.  Thread 0 streams the 18
// chunks through a 3-deep ring (cp.async.bulk completing on "full" mbarriers, refilled when the
// MMAs that read a buffer have completed, which tcgen05.commit signals on its "empty" mbarrier) and
// issues the MMAs of a layer (K = 16 each) into one 128 x 256 FP32 accumulator (256 TMEM columns);
// a commit on the accumulator barrier hands the layer to the epilogue, where each of the 8 warps
// reads half of its 32 rows (TMEM lanes 32 (w % 4) ..) with tcgen05.ld, adds the bias, applies
// tanh and writes the bf16 activations back over the operand tile for the next layer.  112 KB of shared memory and 256 TMEM columns per block:
// two blocks per SM, so one block's epilogue runs beside the other's MMAs and copies.
// Every wait is bounded; a block that gives up records it in the error word, waits (bounded) for
// its own MMAs and copies, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace dg {

namespace {

constexpr int T5_M = 128;                      // positions per block
constexpr int T5_THREADS = 256;                // 8 warps: warps w and w + 4 share TMEM lanes 32 (w % 4) ..
                                               // and take the two 128-column halves of a row
constexpr int T5_NCHUNK = 18;                  // W1, 8 x W2, 8 x W3, W4
constexpr int T5_CHUNK_B = 256 * 32 * 2;       // bytes of a 32-row chunk of a 256-output layer
constexpr int T5_W4_B = 16 * 256 * 2;          // bytes of the packed W4
constexpr int T5_A_B = T5_M * 256 * 2;         // operand tile (activations)
constexpr int T5_NBUF = 3;                     // weight-chunk ring depth
constexpr uint32_t T5_TMEM_COLS = 256;
constexpr long long T5_WAIT = 4000000000LL;    // ~2 s at 2 GHz
constexpr int GIN = 32, GH = 256;
// packed weights: 17 chunks of 8192 bf16 (W1, W2, W3) and 4096 for W4
constexpr int64_t T5_PACKED = 17 * 8192 + 4096;

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(b)), "r"(n) : "memory");
}

__device__ __forceinline__ bool bar_test(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s_addr(b)), "r"(parity), "r"(2000u)
        : "memory");
    return ok != 0;
}

// bounded wait; with `fail` given it also gives up at once when another thread of the block failed
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, volatile int* fail)
{
    long long t0 = clock64();
    while (!bar_test(b, parity)) {
        if (fail && *fail) return false;
        if (clock64() - t0 > T5_WAIT) return false;
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(b)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     s_addr(dst)),
                 "l"(src), "r"(bytes), "r"(s_addr(b))
                 : "memory");
}

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets of the
// core matrices, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(b))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane (asynchronous: tmem_wait before use)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tanh_mufu(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t bf2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// byte offset of element (r, k) in the operand tile (128 rows x 256 K)
__device__ __forceinline__ uint32_t a_off(int r, int k) { return (r >> 3) * 4096 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

}  // namespace

// Pack the bf16 weights (W1 [32][256], W2, W3 [256][256], W4 [256][8] with columns 4..7 zero; the
// layout of the mma.sync kernel) into the transposed chunks of the tcgen05 kernel.
__global__ void k_pack_tc05(const __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wt)
{
    int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= T5_PACKED) return;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    __nv_bfloat16 v = zero;
    if (d < 17 * 8192) {
        // chunk c, 256 outputs x 32 K: (n, kk) at (n / 8) * 512 + (kk / 8) * 128 + (n % 8) * 16 + (kk % 8) * 2 B
        int c = (int)(d / 8192), o = (int)(d % 8192) * 2;
        int nb = o / 512, rem = o % 512, kb = rem / 128, rr = rem % 128;
        int n = nb * 8 + rr / 16, kk = kb * 8 + (rr % 16) / 2;
        if (c == 0) v = wb[kk * GH + n];
        else if (c <= 8) v = wb[GIN * GH + ((c - 1) * 32 + kk) * GH + n];
        else v = wb[GIN * GH + GH * GH + ((c - 9) * 32 + kk) * GH + n];
    } else {
        // W4, 16 outputs x 256 K: (n, k) at (n / 8) * 4096 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2 B
        int o = (int)(d - 17 * 8192) * 2;
        int nb = o / 4096, rem = o % 4096, kb = rem / 128, rr = rem % 128;
        int n = nb * 8 + rr / 16, k = kb * 8 + (rr % 16) / 2;
        if (n < 4) v = wb[GIN * GH + 2 * GH * GH + k * 8 + n];
    }
    wt[d] = v;
}

__global__ void __launch_bounds__(T5_THREADS) k_guess_forward_tc05(int64_t M, const float* __restrict__ X,
                                                                  const __nv_bfloat16* __restrict__ wt,
                                                                  const float* __restrict__ bias1,
                                                                  const float* __restrict__ bias2,
                                                                  const float* __restrict__ bias3,
                                                                  const float* __restrict__ bias4,
                                                                  float* __restrict__ out, const int* gate, int* err)
{
    if (gate && !*gate) return;
    extern __shared__ __align__(128) unsigned char t5_smem[];
    unsigned char* At = t5_smem;                 // operand tile (activations), 64 KB
    unsigned char* Wb = t5_smem + T5_A_B;        // weight-chunk ring, T5_NBUF x 16 KB
    __shared__ uint64_t full[T5_NBUF], empty[T5_NBUF], accb, drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    volatile int* vfail = &fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = (warp & 3) * 32 + (tid & 31);   // accumulator row = TMEM lane of this thread
    const int half = warp >> 2;                     // the 128-column half of the row it takes
    const int64_t m0 = (int64_t)blockIdx.x * T5_M;
    if (tid == 0) {
        for (int b = 0; b < T5_NBUF; b++) {
            bar_init(&full[b], 1);
            bar_init(&empty[b], 1);
        }
        bar_init(&accb, 1);
        bar_init(&drain, 1);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_slot)),
                     "r"(T5_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // input rows -> bf16 operand columns 0..31 (rows past M are zero); each half of the threads
    // converts 16 of the 32 columns
    {
        const int64_t gm = m0 + row;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int kb = 2 * half + q;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (gm < M) {
                a = *reinterpret_cast<const float4*>(X + gm * GIN + kb * 8);
                b = *reinterpret_cast<const float4*>(X + gm * GIN + kb * 8 + 4);
            }
            *reinterpret_cast<uint4*>(At + a_off(row, kb * 8)) =
                make_uint4(bf2(a.x, a.y), bf2(a.z, a.w), bf2(b.x, b.y), bf2(b.z, b.w));
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operand writes -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    // chunk c: source offset and bytes
    auto chunk_src = [&](int c) { return wt + (int64_t)c * 8192; };
    auto chunk_bytes = [&](int c) { return (uint32_t)(c == T5_NCHUNK - 1 ? T5_W4_B : T5_CHUNK_B); };
    int loaded = 0;     // chunks whose copy thread 0 has issued
    int consumed = 0;   // chunks whose MMAs thread 0 has issued
    if (tid == 0) {
        for (; loaded < T5_NBUF - 1; loaded++)
            bulk_g2s(Wb + (loaded % T5_NBUF) * T5_CHUNK_B, chunk_src(loaded), chunk_bytes(loaded),
                     &full[loaded % T5_NBUF]);
    }
    for (int layer = 0; layer < 4; layer++) {
        const int nch = (layer == 0 || layer == 3) ? 1 : 8;
        if (tid == 0 && !*vfail) {
            const uint32_t id = layer == 3 ? idesc_bf16(T5_M, 16) : idesc_bf16(T5_M, 256);
            for (int j = 0; j < nch; j++) {
                const int c = consumed, b = c % T5_NBUF;
                if (!bar_wait(&full[b], (uint32_t)((c / T5_NBUF) & 1), vfail)) { fail = 1; break; }
                tc_fence_after();
                const uint32_t wbase = s_addr(Wb + b * T5_CHUNK_B), abase = s_addr(At);
                if (layer < 3) {
#pragma unroll
                    for (int ks = 0; ks < 2; ks++) {
                        const int kb = 4 * j + 2 * ks;   // the layer's K offset / 8
                        mma(tmem, mdesc(abase + kb * 128, 128, 4096), mdesc(wbase + 2 * ks * 128, 128, 512), id,
                            (j | ks) != 0);
                    }
                } else {
#pragma unroll 4
                    for (int ks = 0; ks < 16; ks++)
                        mma(tmem, mdesc(abase + 2 * ks * 128, 128, 4096), mdesc(wbase + 2 * ks * 128, 128, 4096), id,
                            ks != 0);
                }
                mma_commit(&empty[b]);
                consumed++;
                // refill the buffer of chunk c - 1 (its MMAs, queued before this chunk's, are done
                // when its commit lands) with chunk c + T5_NBUF - 1
                if (loaded < T5_NBUF - 1 + consumed && loaded < T5_NCHUNK) {
                    const int nb = loaded % T5_NBUF;
                    if (loaded >= T5_NBUF &&
                        !bar_wait(&empty[nb], (uint32_t)(((loaded - T5_NBUF) / T5_NBUF) & 1), vfail)) {
                        fail = 1;
                        break;
                    }
                    bulk_g2s(Wb + nb * T5_CHUNK_B, chunk_src(loaded), chunk_bytes(loaded), &full[nb]);
                    loaded++;
                }
            }
            mma_commit(&accb);   // the layer's accumulator is complete when this lands
        }
        // epilogue: this thread's accumulator row (TMEM lane) and column half; the TMEM loads are
        // warp-wide, so the decision to read is made per warp
        bool ok = bar_wait(&accb, (uint32_t)(layer & 1), vfail);
        if (!ok) fail = 1;
        tc_fence_after();
        const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        ok = __all_sync(0xffffffffu, ok && !*vfail);
        if (ok) {
            if (layer < 3) {
                const float* bias = layer == 0 ? bias1 : layer == 1 ? bias2 : bias3;   // warp-uniform reads
#pragma unroll 1
                for (int cb = half * 4; cb < half * 4 + 4; cb++) {   // 32 columns per round
                    uint32_t v[32];
                    tmem_ld16(trow + cb * 32, v);
                    tmem_ld16(trow + cb * 32 + 16, v + 16);
                    tmem_wait();
                    uint32_t p[16];
#pragma unroll
                    for (int j = 0; j < 16; j++)
                        p[j] = bf2(tanh_mufu(__uint_as_float(v[2 * j]) + __ldg(bias + cb * 32 + 2 * j)),
                                   tanh_mufu(__uint_as_float(v[2 * j + 1]) + __ldg(bias + cb * 32 + 2 * j + 1)));
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        *reinterpret_cast<uint4*>(At + a_off(row, cb * 32 + 8 * q)) =
                            make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
                }
            } else if (half == 0) {
                uint32_t v[16];
                tmem_ld16(trow, v);
                tmem_wait();
                const int64_t gm = m0 + row;
                if (gm < M)
                    *reinterpret_cast<float4*>(out + gm * 4) =
                        make_float4(__uint_as_float(v[0]) + __ldg(bias4), __uint_as_float(v[1]) + __ldg(bias4 + 1),
                                    __uint_as_float(v[2]) + __ldg(bias4 + 2), __uint_as_float(v[3]) + __ldg(bias4 + 3));
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (*vfail) break;
    }
    if (*vfail && tid == 0) {
        atomicExch(err, 1);
        // the block's own MMAs and copies still in flight: a commit on the drain barrier lands when
        // every MMA issued so far has completed; each issued copy lands on its buffer's barrier
        mma_commit(&drain);
        bar_wait(&drain, 0, nullptr);
        for (int c = consumed; c < loaded; c++) bar_wait(&full[c % T5_NBUF], (uint32_t)((c / T5_NBUF) & 1), nullptr);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T5_TMEM_COLS) : "memory");
}

size_t guess_forward_tc05_smem() { return (size_t)T5_A_B + (size_t)T5_NBUF * T5_CHUNK_B; }
int64_t guess_tc05_packed() { return T5_PACKED; }
int guess_tc05_rows() { return T5_M; }

cudaError_t guess_tc05_prepare()
{
    return cudaFuncSetAttribute(k_guess_forward_tc05, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)guess_forward_tc05_smem());
}

void launch_pack_tc05(cudaStream_t st, const __nv_bfloat16* wb, __nv_bfloat16* wt)
{
    k_pack_tc05<<<(unsigned)((T5_PACKED + 255) / 256), 256, 0, st>>>(wb, wt);
}

void launch_guess_forward_tc05(cudaStream_t st, int64_t M, const float* X, const __nv_bfloat16* wt,
                               const float* b1, const float* b2, const float* b3, const float* b4, float* out,
                               const int* gate, int* err)
{
    if (M <= 0) return;
    k_guess_forward_tc05<<<(unsigned)((M + T5_M - 1) / T5_M), T5_THREADS, guess_forward_tc05_smem(), st>>>(
        M, X, wt, b1, b2, b3, b4, out, gate, err);
}

}  // namespace dg
