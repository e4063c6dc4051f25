// guess_tc05.cu -- forward pass of the learned initial-guess network (32 -> 256 -> 256 -> 256 -> 4,
// tanh; bf16 weights and activations, FP32 accumulation) on the fifth-generation tensor cores:
// tcgen05.mma with the accumulators in tensor memory (TMEM).
//
// Tile = 128 positions = one MMA tile (M = 128).  The tile's activations live in shared memory as
// bf16 in the K-major, no-swizzle operand layout of the MMA (8 x 8 core matrices of 128 B;
// element (r, k) at (k / 8) * 2048 + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2 bytes).  The
// transposed weights are packed once per parameter update into the same layout, in 16 KB chunks of
// 32 K-rows x 256 outputs (W1: 1 chunk, W2 and W3: 8 each, W4: one 8 KB chunk of 256 K x 16
// outputs, columns 4..15 zero), so a chunk is one contiguous bulk copy.
//
// One persistent block per SM runs its tiles through a warp-specialised pipeline:
//  - warp 16 (one thread) loads a whole layer's weights (up to 8 chunks, 128 KB) with cp.async.bulk
//    into 8 buffers ("full" mbarrier per buffer) and issues the layer's MMAs (K = 16 each).  A
//    tcgen05.commit drains the tensor pipe, so there is one per layer: it marks the layer's
//    accumulator complete and, with it, its weight buffers free, and the next layer's weights are
//    loaded at once (they land while the epilogue runs).  The layers alternate between two
//    128 x 256 FP32 accumulators in TMEM (512 columns);
//  - warps 0..15 are the epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its 32 rows) of the
//    finished accumulator with tcgen05.ld, adds the bias, applies tanh and writes bf16 activations
//    over the operand tile, one 32-column block at a time (warps 4 h .. 4 h + 3 the blocks h and
//    h + 4).  Each block has an mbarrier that its four warps arrive on, and the next layer's MMAs
//    over that K range are issued as soon as it completes, so they run beside the rest of the
//    epilogue in the other accumulator.  The next tile's input is read into registers early and
//    written once the last layer's MMAs have read the operand tile.
// Every wait is bounded; a block that gives up records it in the error word, waits (bounded) for
// its own MMAs and copies, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace dg {

namespace {

constexpr int T5_M = 128;                      // positions per tile
constexpr int T5_EGRP = 4;                     // epilogue warp groups (4 warps each, one per TMEM lane quadrant)
constexpr int T5_THREADS = (4 * T5_EGRP + 1) * 32;   // 16 epilogue warps + the producer / MMA warp
constexpr int T5_PRODUCER = 4 * T5_EGRP;       // the producer's warp index
constexpr int T5_CHUNK_B = 256 * 32 * 2;       // bytes of a 32-row chunk of a 256-output layer
constexpr int T5_W4_B = 16 * 256 * 2;          // bytes of the packed W4
constexpr int T5_A_B = T5_M * 256 * 2;         // operand tile (activations)
constexpr int T5_NBUF = 8;                     // weight-chunk buffers: one whole layer
constexpr uint32_t T5_TMEM_COLS = 512;         // two 256-column accumulators
constexpr long long T5_WAIT = 4000000000LL;    // ~2 s at 2 GHz
constexpr int GIN = 32, GH = 256;
// packed weights: 17 chunks of 8192 bf16 (W1, W2, W3) and 4096 for W4
constexpr int64_t T5_PACKED = 17 * 8192 + 4096;

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(b)), "r"(n) : "memory");
}

// non-blocking test of a phase; the waits below poll it
__device__ __forceinline__ bool bar_test(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; with `fail` given it also gives up at once when another thread of the block failed.
// backoff_ns > 0: sleep that long between polls (warps whose issue slots others can use)
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, volatile int* fail, unsigned backoff_ns = 0)
{
    long long t0 = clock64();
    while (!bar_test(b, parity)) {
        if (fail && *fail) return false;
        if (clock64() - t0 > T5_WAIT) return false;
        if (backoff_ns) __nanosleep(backoff_ns);
    }
    return true;
}

__device__ __forceinline__ void bar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(b)) : "memory");
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
__device__ __forceinline__ uint32_t a_off(int r, int k) { return (k >> 3) * 2048 + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

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
        // chunk c, 256 outputs x 32 K: (n, kk) at (kk / 8) * 4096 + (n / 8) * 128 + (n % 8) * 16 + (kk % 8) * 2 B
        int c = (int)(d / 8192), o = (int)(d % 8192) * 2;
        int kb = o / 4096, rem = o % 4096, nb = rem / 128, rr = rem % 128;
        int n = nb * 8 + rr / 16, kk = kb * 8 + (rr % 16) / 2;
        if (c == 0) v = wb[kk * GH + n];
        else if (c <= 8) v = wb[GIN * GH + ((c - 1) * 32 + kk) * GH + n];
        else v = wb[GIN * GH + GH * GH + ((c - 9) * 32 + kk) * GH + n];
    } else {
        // W4, 16 outputs x 256 K: (n, k) at (k / 8) * 256 + (n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2 B
        int o = (int)(d - 17 * 8192) * 2;
        int kb = o / 256, rem = o % 256, nb = rem / 128, rr = rem % 128;
        int n = nb * 8 + rr / 16, k = kb * 8 + (rr % 16) / 2;
        if (n < 4) v = wb[GIN * GH + 2 * GH * GH + k * 8 + n];
    }
    wt[d] = v;
}

__global__ void __launch_bounds__(T5_THREADS, 1) k_guess_forward_tc05(int64_t M, const float* __restrict__ X,
                                                                     const __nv_bfloat16* __restrict__ wt,
                                                                     const float* __restrict__ bias1,
                                                                     const float* __restrict__ bias2,
                                                                     const float* __restrict__ bias3,
                                                                     const float* __restrict__ bias4,
                                                                     float* __restrict__ out, const int* gate,
                                                                     int* err)
{
    if (gate && !*gate) return;
    extern __shared__ __align__(128) unsigned char t5_smem[];
    unsigned char* At = t5_smem;                 // operand tile (activations), 64 KB
    unsigned char* Wb = t5_smem + T5_A_B;        // one layer's weight chunks, T5_NBUF x 16 KB
    __shared__ uint64_t full[T5_NBUF], accf[2], ardy[8], drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    volatile int* vfail = &fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (M + T5_M - 1) / T5_M;
    if (tid == 0) {
        for (int b = 0; b < T5_NBUF; b++) bar_init(&full[b], 1);
        bar_init(&accf[0], 1);
        bar_init(&accf[1], 1);
        for (int j = 0; j < 8; j++) bar_init(&ardy[j], 4);   // the four warps (one per lane quadrant) of a block
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
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    int nload[T5_NBUF] = {0, 0, 0, 0, 0, 0, 0, 0};   // copies issued into each buffer (producer)
    int nwait[T5_NBUF] = {0, 0, 0, 0, 0, 0, 0, 0};   // ... and waited for
    const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    if (warp == T5_PRODUCER) {
        if (lane == 0) {
            // ---- producer and MMA issuer ----
            auto load_layer = [&](int L) {   // chunks of layer L into buffers 0 ..
                const int c0 = L == 0 ? 0 : L == 1 ? 1 : L == 2 ? 9 : 17, nch = (L == 0 || L == 3) ? 1 : 8;
                for (int j = 0; j < nch; j++) {
                    bulk_g2s(Wb + j * T5_CHUNK_B, wt + (int64_t)(c0 + j) * 8192, L == 3 ? T5_W4_B : T5_CHUNK_B,
                             &full[j]);
                    nload[j]++;
                }
            };
            int nrdy[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // completions of each block barrier consumed
            const uint32_t id256 = idesc_bf16(T5_M, 256), id16 = idesc_bf16(T5_M, 16);
            const uint32_t abase = s_addr(At);
            if (my_tiles > 0) load_layer(0);
            for (int64_t it = 0; it < my_tiles && !*vfail; it++) {
                for (int L = 0; L < 4 && !*vfail; L++) {
                    const int g = (int)(4 * it + L);
                    const uint32_t acc = tmem + (uint32_t)((g & 1) * 256);
                    if (L < 3) {
                        const int nch = L == 0 ? 1 : 8;
                        for (int j = 0; j < nch; j++) {
                            // the chunk's weights and the operand columns 32 j .. 32 j + 31 of the layer's input
                            if (!bar_wait(&full[j], (uint32_t)(nwait[j] & 1), vfail) ||
                                !bar_wait(&ardy[j], (uint32_t)(nrdy[j] & 1), vfail)) {
                                fail = 1;
                                break;
                            }
                            nwait[j]++;
                            nrdy[j]++;
                            tc_fence_after();
                            const uint32_t wbase = s_addr(Wb + j * T5_CHUNK_B);
#pragma unroll
                            for (int ks = 0; ks < 2; ks++)
                                mma(acc, mdesc(abase + (4 * j + 2 * ks) * 2048, 2048, 128),
                                    mdesc(wbase + 2 * ks * 4096, 4096, 128), id256, (j | ks) != 0);
                        }
                    } else {
                        if (!bar_wait(&full[0], (uint32_t)(nwait[0] & 1), vfail)) fail = 1;
                        nwait[0]++;
                        const uint32_t wbase = s_addr(Wb);
                        for (int jj = 0; jj < 8 && !*vfail; jj++) {
                            if (!bar_wait(&ardy[jj], (uint32_t)(nrdy[jj] & 1), vfail)) { fail = 1; break; }
                            nrdy[jj]++;
                            tc_fence_after();
#pragma unroll
                            for (int ks = 2 * jj; ks < 2 * jj + 2; ks++)
                                mma(acc, mdesc(abase + 2 * ks * 2048, 2048, 128), mdesc(wbase + 2 * ks * 256, 256, 128),
                                    id16, ks != 0);
                        }
                    }
                    if (*vfail) break;
                    mma_commit(&accf[g & 1]);   // accumulator complete, weight buffers free
                    // the next layer's weights replace this layer's once its MMAs have completed
                    const bool more = L < 3 || it + 1 < my_tiles;
                    if (more) {
                        if (!bar_wait(&accf[g & 1], (uint32_t)((g >> 1) & 1), vfail)) { fail = 1; break; }
                        load_layer((L + 1) & 3);
                    }
                }
            }
        }
    } else {
        // ---- epilogue warps ----
        const int row = (warp & 3) * 32 + lane;     // accumulator row = TMEM lane of this thread
        const int grp = warp >> 2;                  // column blocks grp, grp + T5_EGRP, ...
        const uint32_t tl = (uint32_t)((warp & 3) * 32) << 16;
        float4 xr[8];                               // the next tile's input row (warps 0..3)
        auto read_x = [&](int64_t tile) {
            const int64_t gm = tile * T5_M + row;
#pragma unroll
            for (int q = 0; q < 8; q++)
                xr[q] = gm < M ? *reinterpret_cast<const float4*>(X + gm * GIN + q * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        auto write_x = [&]() {                      // input row -> operand block 0, then release it
#pragma unroll
            for (int kb = 0; kb < GIN / 8; kb++)
                *reinterpret_cast<uint4*>(At + a_off(row, kb * 8)) =
                    make_uint4(bf2(xr[2 * kb].x, xr[2 * kb].y), bf2(xr[2 * kb].z, xr[2 * kb].w),
                               bf2(xr[2 * kb + 1].x, xr[2 * kb + 1].y), bf2(xr[2 * kb + 1].z, xr[2 * kb + 1].w));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // -> tensor-core reads
            __syncwarp();
            if (lane == 0) bar_arrive(&ardy[0]);
        };
        int64_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
            if (it == 0 && grp == 0) {
                read_x(tile);
                write_x();
            }
            for (int L = 0; L < 4; L++) {
                const int g = (int)(4 * it + L);
                bool ok = bar_wait(&accf[g & 1], (uint32_t)((g >> 1) & 1), vfail, 32);
                if (!ok) fail = 1;
                ok = __all_sync(0xffffffffu, ok && !*vfail);
                if (!ok) break;
                tc_fence_after();
                if (L == 0 && grp == 0 && tile + gridDim.x < ntiles) read_x(tile + gridDim.x);   // lands meanwhile
                const uint32_t acc = tmem + tl + (uint32_t)((g & 1) * 256);
                if (L < 3) {
                    const float* bias = L == 0 ? bias1 : L == 1 ? bias2 : bias3;   // warp-uniform reads
#pragma unroll 1
                    for (int cb = grp; cb < 8; cb += T5_EGRP) {
                        uint32_t v[32];
                        tmem_ld16(acc + cb * 32, v);
                        tmem_ld16(acc + cb * 32 + 16, v + 16);
                        float4 bq[8];   // the block's 32 biases
#pragma unroll
                        for (int q = 0; q < 8; q++) bq[q] = __ldg(reinterpret_cast<const float4*>(bias + cb * 32) + q);
                        const float* bb = reinterpret_cast<const float*>(bq);
                        tmem_wait();
                        uint32_t p[16];
#pragma unroll
                        for (int j = 0; j < 16; j++)
                            p[j] = bf2(tanh_mufu(__uint_as_float(v[2 * j]) + bb[2 * j]),
                                       tanh_mufu(__uint_as_float(v[2 * j + 1]) + bb[2 * j + 1]));
#pragma unroll
                        for (int q = 0; q < 4; q++)
                            *reinterpret_cast<uint4*>(At + a_off(row, cb * 32 + 8 * q)) =
                                make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) bar_arrive(&ardy[cb]);
                    }
                } else {
                    // the last layer's MMAs have read the operand tile: the next tile's input first
                    // (it lets the next tile's first MMAs start), then this tile's outputs
                    if (grp == 0 && tile + gridDim.x < ntiles) write_x();
                    if (grp == 0) {
                        uint32_t v[16];
                        tmem_ld16(acc, v);
                        tmem_wait();
                        const int64_t gm = tile * T5_M + row;
                        if (gm < M)
                            *reinterpret_cast<float4*>(out + gm * 4) = make_float4(
                                __uint_as_float(v[0]) + __ldg(bias4), __uint_as_float(v[1]) + __ldg(bias4 + 1),
                                __uint_as_float(v[2]) + __ldg(bias4 + 2), __uint_as_float(v[3]) + __ldg(bias4 + 3));
                    }
                    tc_fence_before();
                }
            }
            if (*vfail) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (*vfail && tid == T5_PRODUCER * 32) {
        atomicExch(err, 1);
        // the block's own MMAs and copies still in flight: a commit on the drain barrier lands when
        // every MMA issued so far has completed; each issued copy lands on its buffer's barrier
        mma_commit(&drain);
        bar_wait(&drain, 0, nullptr);
        for (int j = 0; j < T5_NBUF; j++)
            for (; nwait[j] < nload[j]; nwait[j]++) bar_wait(&full[j], (uint32_t)(nwait[j] & 1), nullptr);
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
    static int nsm = 0;   // persistent blocks: one per SM (a block takes all of an SM's TMEM)
    if (!nsm) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
            nsm = 1;
    }
    const int64_t ntiles = (M + T5_M - 1) / T5_M;
    const unsigned grid = (unsigned)(ntiles < nsm ? ntiles : nsm);
    k_guess_forward_tc05<<<grid, T5_THREADS, guess_forward_tc05_smem(), st>>>(M, X, wt, b1, b2, b3, b4, out, gate,
                                                                           err);
}

}  // namespace dg
