// mlp_kernels.cu -- BF16 tensor-core kernels of the crater-surrogate MLP (5 -> 4 x 256 GELU
// -> 66) and its training step.
//
// One GEMM kernel serves every contraction of the forward and backward passes:
//     C[m][n] = sum_k A(m, k) B(n, k),   A(m, k) = A[m a_sm + k a_sk],  B(n, k) = B[n b_sn + k b_sk]
// with BF16 operands and an FP32 accumulator.  A CTA owns a 128 x NT tile of C (NT <= 128, a
// multiple of 16).  Its 128 threads gather 128 x 64 and NT x 64 operand tiles from global
// memory (any strides, zero outside the matrix) into shared memory in the tensor cores'
// canonical K-major layout without swizzle: 8-row x 16-byte core matrices, 128 bytes each,
// adjacent along M/N (stride 128 B) and then along K (stride rows x 16 B).  One elected
// thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128, N = NT, K = 16) four
// times per 64-wide K slice, accumulating in tensor memory; tcgen05.commit arrives on the
// stage's mbarrier when those MMAs have read their operands, which frees the stage for the
// next gather (two stages).  The epilogue reads the accumulator back with tcgen05.ld (warp w
// owns TMEM lanes 32w..32w+31, i.e. rows 32w..32w+31 of the tile) and applies one of the
// fused operations below.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records an error code, waits
// (bounded again) for its own MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp_internal.cuh"

namespace salec {
namespace mlp {

constexpr int kBM = 128;          // rows of a C tile = TMEM lanes
constexpr int kBK = 64;           // K slice per stage
constexpr int kGemmThreads = 128;
constexpr int kMaxNT = 128;       // widest C tile (columns = TMEM columns)
constexpr unsigned long long kWaitNs = 2000000000ull;   // a wait on an mbarrier fails after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of tcgen05: start address, leading-dimension byte offset
// (between core matrices adjacent along K), stride-dimension byte offset (between core
// matrices adjacent along M/N), the fixed field 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// bounded wait; false when the time limit ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// Gather 8 consecutive-in-k elements of row r into one 16-byte core-matrix row.
__device__ __forceinline__ uint4 gather8(const __nv_bfloat16* __restrict__ P, long s_r, long s_k, int r, int R, int k0,
                                         int K)
{
    union { uint4 u; __nv_bfloat16 h[8]; } w;
    if (r < R && s_k == 1 && k0 + 8 <= K && ((reinterpret_cast<uintptr_t>(P + r * s_r + k0) & 15) == 0)) {
        w.u = *reinterpret_cast<const uint4*>(P + r * s_r + k0);
        return w.u;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = k0 + e;
        w.h[e] = (r < R && k < K) ? P[r * s_r + (long)k * s_k] : __float2bfloat16_rn(0.0f);
    }
    return w.u;
}

__global__ void __launch_bounds__(kGemmThreads) k_gemm_bf16(GemmArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // stage s: A tile at s * stage_bytes, B tile right after it
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tmem_holder;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * g.nt;
    const int NT = g.nt;
    const uint32_t a_bytes = kBM * kBK * 2, b_bytes = (uint32_t)NT * kBK * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    const uint32_t tmem_cols = g.tmem_cols;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;
    const uint32_t idesc = idesc_bf16(kBM, NT);

    const int nk = (g.K + kBK - 1) / kBK;
    bool ok = true;
    int issued = 0;                       // K slices whose MMAs were committed
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt & 1;
        // uniform decision: a barrier whose result every thread sees
        if (kt >= 2 && !__syncthreads_and(mbar_wait(&bars[s], ((kt - 2) >> 1) & 1))) { ok = false; break; }
        unsigned char* sa = smem + s * stage_bytes;
        unsigned char* sb = sa + a_bytes;
        const int k0 = kt * kBK;
        // A: thread tid gathers row tid; core matrix (row group rg, k group kg) at kg*2048 + rg*128
#pragma unroll
        for (int kg = 0; kg < 8; ++kg) {
            const uint4 w = gather8(g.A, g.a_sm, g.a_sk, m0 + tid, g.M, k0 + 8 * kg, g.K);
            *reinterpret_cast<uint4*>(sa + kg * (kBM * 16) + (tid >> 3) * 128 + (tid & 7) * 16) = w;
        }
        for (int r = tid; r < NT; r += kGemmThreads) {
#pragma unroll
            for (int kg = 0; kg < 8; ++kg) {
                const uint4 w = gather8(g.B, g.b_sn, g.b_sk, n0 + r, g.N, k0 + 8 * kg, g.K);
                *reinterpret_cast<uint4*>(sb + kg * (NT * 16) + (r >> 3) * 128 + (r & 7) * 16) = w;
            }
        }
        // generic-proxy writes -> visible to the tensor cores' (async proxy) reads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
                // K = 16 spans two core matrices along K
                const uint64_t ad = sdesc(a0 + kk * 2 * (kBM * 16), kBM * 16, 128);
                const uint64_t bd = sdesc(b0 + kk * 2 * (NT * 16), NT * 16, 128);
                mma_bf16(tmem, ad, bd, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&bars[s]);
        }
        issued = kt + 1;
    }
    // all MMAs done: wait for the last commit of each stage (the later one covers every
    // earlier MMA; waiting for both leaves no arrive pending when the CTA exits)
    if (ok && issued >= 2) ok = __syncthreads_and(mbar_wait(&bars[(issued - 2) & 1], ((issued - 2) >> 1) & 1));
    if (ok && issued >= 1) ok = __syncthreads_and(mbar_wait(&bars[(issued - 1) & 1], ((issued - 1) >> 1) & 1));
    if (!ok) {
        if (g.err && tid == 0) atomicOr(g.err, 1);
        // give MMAs still in flight a bounded chance to finish before their memory goes away
        if (issued >= 1) (void)mbar_wait(&bars[(issued - 1) & 1], ((issued - 1) >> 1) & 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (ok) {
        const int m = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        double lsum = 0.0;
        for (int c0 = 0; c0 < NT; c0 += 16) {
            float v[16];
            tmem_ld16(trow + (uint32_t)c0, v);
            if (m >= g.M) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = n0 + c0 + j;
                if (n >= g.N) break;
                float x = nk > 0 ? v[j] : 0.0f;    // K = 0: empty sum
                switch (g.epi) {
                case kEpiStore:
                    if (g.bias) x += g.bias[n];
                    g.C[(long)m * g.ldc + n] = x;
                    break;
                case kEpiBiasGelu: {
                    x += g.bias[n];
                    g.C[(long)m * g.ldc + n] = x;                                   // Z
                    g.Hout[(long)m * g.ldh + n] = __float2bfloat16_rn(gelu_f(x));   // gelu(Z)
                    break;
                }
                case kEpiGeluBwd: {
                    const float z = g.Zin[(long)m * g.ldz + n];
                    g.Hout[(long)m * g.ldh + n] = __float2bfloat16_rn(x * gelu_grad_f(z));
                    break;
                }
                case kEpiOutLoss: {
                    x += g.bias[n];
                    g.C[(long)m * g.ldc + n] = x;                                   // Y
                    const float d = x - g.Tin[(long)m * g.ldt + n];
                    lsum += (double)d * (double)d;
                    g.Hout[(long)m * g.ldh + n] = __float2bfloat16_rn(d * g.grad_scale);
                    break;
                }
                }
            }
        }
        if (g.epi == kEpiOutLoss && g.loss) {
            for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
            if (lane == 0 && lsum != 0.0) atomicAdd(g.loss, lsum);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// Column sums of a BF16 matrix (bias gradients): out[n] = sum_m G[m][n].
__global__ void k_colsum(const __nv_bfloat16* __restrict__ G, int M, int N, long ldg, float* __restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int m = 0; m < M; ++m) s += __bfloat162float(G[(long)m * ldg + n]);
    out[n] = s;
}

// FP32 -> BF16 (inputs of the first layer).
__global__ void k_to_bf16(const float* __restrict__ x, long n, __nv_bfloat16* __restrict__ y)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// Adam on the FP32 master parameters; refreshes the BF16 copy of every weight.  wmap[i] is
// the index of parameter i in the BF16 weight block, or -1 for a bias.
__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m1, float* __restrict__ m2,
                       const float* __restrict__ grad, long n, AdamArgs a, const int* __restrict__ wmap,
                       __nv_bfloat16* __restrict__ wbf)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = a.beta1 * m1[i] + (1.0f - a.beta1) * g;
    const float vi = a.beta2 * m2[i] + (1.0f - a.beta2) * g * g;
    m1[i] = mi;
    m2[i] = vi;
    const float th = theta[i] - a.lr * (mi * a.c1) / (sqrtf(vi * a.c2) + a.eps);
    theta[i] = th;
    const int w = wmap[i];
    if (w >= 0) wbf[w] = __float2bfloat16_rn(th);
}

// BF16 copy of the weights from the FP32 parameters.
__global__ void k_refresh_bf16(const float* __restrict__ theta, long n, const int* __restrict__ wmap,
                               __nv_bfloat16* __restrict__ wbf)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int w = wmap[i];
    if (w >= 0) wbf[w] = __float2bfloat16_rn(theta[i]);
}

size_t gemm_smem_bytes(int nt) { return 2 * (size_t)(kBM * kBK * 2 + nt * kBK * 2) + 1024; }

cudaError_t launch_gemm(const GemmArgs& g0, cudaStream_t s)
{
    GemmArgs g = g0;
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    const int nt = ((g.N < kMaxNT ? g.N : kMaxNT) + 15) / 16 * 16;
    g.nt = nt;
    int cols = 32;
    while (cols < nt) cols <<= 1;
    g.tmem_cols = cols;
    const size_t smem = gemm_smem_bytes(nt);
    // the attribute is per device
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem_bytes(kMaxNT));
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    dim3 grid((unsigned)((g.M + kBM - 1) / kBM), (unsigned)((g.N + nt - 1) / nt));
    k_gemm_bf16<<<grid, kGemmThreads, smem, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_colsum(const __nv_bfloat16* G, int M, int N, long ldg, float* out, cudaStream_t s)
{
    k_colsum<<<(N + 127) / 128, 128, 0, s>>>(G, M, N, ldg, out);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* x, long n, __nv_bfloat16* y, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, y);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, float* m1, float* m2, const float* grad, long n, const AdamArgs& a,
                        const int* wmap, __nv_bfloat16* wbf, cudaStream_t s)
{
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(theta, m1, m2, grad, n, a, wmap, wbf);
    return cudaGetLastError();
}

cudaError_t launch_refresh_bf16(const float* theta, long n, const int* wmap, __nv_bfloat16* wbf, cudaStream_t s)
{
    k_refresh_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(theta, n, wmap, wbf);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace salec
