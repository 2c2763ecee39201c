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
// Operands that are K-major rows of 16-byte multiples (the forward pass) take a second
// kernel, k_gemm_bf16_tma, fed by TMA (below).
//
// Every wait on an mbarrier is bounded; on expiry the kernel records an error code, waits
// (bounded again) for its own MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp_internal.cuh"
#include "salec_tma.cuh"

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

// The normal CDF Phi(z) = (1 + erf(z / sqrt 2)) / 2, with the complementary error function
// of Abramowitz & Stegun, Handbook of Mathematical Functions, formula 7.1.26: for x >= 0,
// erfc(x) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2) + e(x), t = 1 / (1 + p x),
// |e(x)| <= 1.5e-7.  Phi(z) is 1 - erfc(x) / 2 for z >= 0 and erfc(x) / 2 for z < 0
// (x = |z| / sqrt 2), so the left tail is formed without cancellation.  Also returns
// exp(-z^2 / 2) (the same exponential), which the GELU derivative needs.  The error is far
// below the BF16 rounding (2^-9 relative) that every activation goes through.
__device__ __forceinline__ float normal_cdf(float z, float* gauss)
{
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    float pol = fmaf(t, 1.061405429f, -1.453152027f);
    pol = fmaf(t, pol, 1.421413741f);
    pol = fmaf(t, pol, -0.284496736f);
    pol = fmaf(t, pol, 0.254829592f);
    const float e = __expf(-x * x);
    *gauss = e;
    const float half_erfc = 0.5f * (pol * t) * e;
    return z >= 0.0f ? 1.0f - half_erfc : half_erfc;
}

// The same GELU for two values at once: every multiply and multiply-add issues as one
// packed FP32x2 instruction (each lane rounded as the scalar instruction would), the
// reciprocal and the exponential as the hardware approximations the scalar form uses, in
// the same order, so the results are those of gelu_f.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2(float a, float b) { return (f32x2)__float_as_uint(a) | ((f32x2)__float_as_uint(b) << 32); }
__device__ __forceinline__ float f2lo(f32x2 v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float f2hi(f32x2 v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ f32x2 f2mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 f2add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 gelu_pair(f32x2 z)
{
    const float z0 = f2lo(z), z1 = f2hi(z);
    const f32x2 x = f2mul(f2(fabsf(z0), fabsf(z1)), f2(0.70710678118654752f, 0.70710678118654752f));
    const f32x2 d = f2fma(f2(0.3275911f, 0.3275911f), x, f2(1.0f, 1.0f));
    const f32x2 t = f2(__fdividef(1.0f, f2lo(d)), __fdividef(1.0f, f2hi(d)));
    f32x2 pol = f2fma(t, f2(1.061405429f, 1.061405429f), f2(-1.453152027f, -1.453152027f));
    pol = f2fma(t, pol, f2(1.421413741f, 1.421413741f));
    pol = f2fma(t, pol, f2(-0.284496736f, -0.284496736f));
    pol = f2fma(t, pol, f2(0.254829592f, 0.254829592f));
    const f32x2 nx2 = f2mul(f2(-f2lo(x), -f2hi(x)), x);
    const f32x2 e = f2(__expf(f2lo(nx2)), __expf(f2hi(nx2)));
    const f32x2 h = f2mul(f2mul(f2(0.5f, 0.5f), f2mul(pol, t)), e);
    const float P0 = z0 >= 0.0f ? 1.0f - f2lo(h) : f2lo(h);
    const float P1 = z1 >= 0.0f ? 1.0f - f2hi(h) : f2hi(h);
    return f2mul(z, f2(P0, P1));
}

// GELU in its erf form, z Phi(z), and its derivative Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_f(float z)
{
    float e;
    return z * normal_cdf(z, &e);
}
__device__ __forceinline__ float gelu_grad_f(float z)
{
    float e;
    const float P = normal_cdf(z, &e);
    return fmaf(z * 0.39894228040143268f, e, P);
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

// Epilogue: warp w reads TMEM lanes 32w..32w+31 (rows m0 + 32w + lane of the tile), 16
// columns at a time, and applies the fused operation of g.epi.  In kEpiBiasGelu a null C
// skips the pre-activation store (inference).  A row's 16 columns go out as 16-byte stores
// when they lie inside N and the rows are 16-byte aligned (each thread writes its own row:
// whole sectors, merged in L2); otherwise element by element.
__device__ __forceinline__ void epilogue(const GemmArgs& g, uint32_t tmem, int m0, int n0, int NT, bool any_k)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    double lsum = 0.0;
    const bool vec_c = !g.Cb && ((g.ldc * 4) & 15) == 0 && ((reinterpret_cast<uintptr_t>(g.C) & 15) == 0);
    const bool vec_h = ((g.ldh * 2) & 15) == 0 && ((reinterpret_cast<uintptr_t>(g.Hout) & 15) == 0);
    const bool has_c = g.epi != kEpiGeluBwd && g.C != nullptr;
    const bool has_h = g.epi != kEpiStore;
    for (int c0 = 0; c0 < NT; c0 += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c0, v);
        if (m >= g.M) continue;
        const int nb = n0 + c0;
        const bool full = nb + 16 <= g.N;
        float x[16], h[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int n = nb + j;
            const bool in = full || n < g.N;
            float y = any_k ? v[j] : 0.0f;    // K = 0: empty sum
            h[j] = 0.0f;
            switch (g.epi) {
            case kEpiStore:
                if (g.bias && in) y += g.bias[n];
                break;
            case kEpiBiasGelu:
                if (in) y += g.bias[n];
                h[j] = gelu_f(y);
                break;
            case kEpiGeluBwd:
                h[j] = in ? y * gelu_grad_f(g.Zin[(long)m * g.ldz + n]) : 0.0f;
                break;
            case kEpiOutLoss:
                if (in) {
                    y += g.bias[n];
                    const float d = y - g.Tin[(long)m * g.ldt + n];
                    lsum += (double)d * (double)d;
                    h[j] = d * g.grad_scale;
                }
                break;
            }
            x[j] = y;
        }
        if (full && has_c && vec_c) {
            float4* dst = reinterpret_cast<float4*>(g.C + (long)m * g.ldc + nb);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
        } else if (has_c) {
            for (int j = 0; j < 16 && nb + j < g.N; ++j) {
                if (g.Cb && nb + j == g.N - 1)
                    g.Cb[m] = x[j];          // the column of the row of ones: a bias gradient
                else
                    g.C[(long)m * g.ldc + nb + j] = x[j];
            }
        }
        if (full && has_h && vec_h) {
            union { uint4 u[2]; __nv_bfloat16 b[16]; } pk;
#pragma unroll
            for (int j = 0; j < 16; ++j) pk.b[j] = __float2bfloat16_rn(h[j]);
            uint4* dst = reinterpret_cast<uint4*>(g.Hout + (long)m * g.ldh + nb);
            dst[0] = pk.u[0];
            dst[1] = pk.u[1];
        } else if (has_h) {
            for (int j = 0; j < 16 && nb + j < g.N; ++j) g.Hout[(long)m * g.ldh + nb + j] = __float2bfloat16_rn(h[j]);
        }
        // the transposed copy: for each column, the warp's 32 rows are 64 contiguous bytes
        if (has_h && g.HoutT) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (full || nb + j < g.N) g.HoutT[(long)(nb + j) * g.ldhT + m] = __float2bfloat16_rn(h[j]);
        }
    }
    if (g.epi == kEpiOutLoss && g.loss) {
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
        if (lane == 0 && lsum != 0.0) atomicAdd(g.loss, lsum);
    }
}

__global__ void __launch_bounds__(kGemmThreads) k_gemm_bf16(GemmArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // stage s: A tile at s * stage_bytes, B tile right after it
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tmem_holder;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * g.nt;
    const int NT = g.nt;
    // split-K: this CTA sums K range [kb, ke) into its own partial (plain store); a
    // second kernel adds the partials in a fixed order
    const int kb = g.kchunk > 0 ? (int)blockIdx.z * g.kchunk : 0;
    const int ke = g.kchunk > 0 ? min(g.K, kb + g.kchunk) : g.K;
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

    const int nk = (ke - kb + kBK - 1) / kBK;
    bool ok = true;
    int issued = 0;                       // K slices whose MMAs were committed
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt & 1;
        // uniform decision: a barrier whose result every thread sees
        if (kt >= 2 && !__syncthreads_and(mbar_wait(&bars[s], ((kt - 2) >> 1) & 1))) { ok = false; break; }
        unsigned char* sa = smem + s * stage_bytes;
        unsigned char* sb = sa + a_bytes;
        const int k0 = kb + kt * kBK;
        // A: thread tid gathers row tid; core matrix (row group rg, k group kg) at kg*2048 + rg*128
#pragma unroll
        for (int kg = 0; kg < 8; ++kg) {
            const uint4 w = gather8(g.A, g.a_sm, g.a_sk, m0 + tid, g.M, k0 + 8 * kg, ke);
            *reinterpret_cast<uint4*>(sa + kg * (kBM * 16) + (tid >> 3) * 128 + (tid & 7) * 16) = w;
        }
        for (int r = tid; r < NT; r += kGemmThreads) {
#pragma unroll
            for (int kg = 0; kg < 8; ++kg) {
                const uint4 w = gather8(g.B, g.b_sn, g.b_sk, n0 + r, g.N, k0 + 8 * kg, ke);
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
        if (g.kchunk > 0) {
            GemmArgs gp = g;
            gp.C = g.part + (long)blockIdx.z * g.M * g.N;
            gp.ldc = g.N;
            gp.Cb = nullptr;
            epilogue(gp, tmem, m0, n0, NT, nk > 0);
        } else {
            epilogue(g, tmem, m0, n0, NT, nk > 0);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// ---------------------------------------------------------------------------------------
// The same contraction when both operands are K-major rows (A[m][k], B[n][k], rows of
// 16-byte multiples): the forward pass.  One thread streams K slices into a ring of
// kStages shared-memory stages with TMA (cp.async.bulk.tensor, 2-D maps, boxes of 8
// elements x rows: one box is one column of core matrices, 16 bytes x rows, exactly the
// canonical no-swizzle K-major layout), each stage's mbarrier completing on the bytes
// delivered; the same thread issues the MMAs of a slice as soon as it lands and refills
// the stage once tcgen05.commit reports those MMAs done.  The tile is 128 x NT with NT up
// to 256 (a whole hidden layer, so the activations are read once).
// ---------------------------------------------------------------------------------------
constexpr int kStages = 4;
constexpr int kMaxNT_TMA = 256;

// One GEMM for each member of an ensemble, launched together: the members' tensor maps and
// arguments (the same shapes and plan, their own buffers).
struct GroupGemm {
    CUtensorMap ma[kMaxGroup], mb[kMaxGroup];
    GemmArgs g[kMaxGroup];
    int n, S;
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// The body of the TMA-fed GEMM for one CTA: its tile (blockIdx.x, blockIdx.y) of the product
// that g describes, K split `zsplit` of it.
__device__ __forceinline__ void gemm_tma_body(const CUtensorMap* mapA_p, const CUtensorMap* mapB_p, const GemmArgs& g,
                                              int zsplit)
{
    const CUtensorMap& mapA = *mapA_p;
    const CUtensorMap& mapB = *mapB_p;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t full[kStages], empty[kStages];
    __shared__ uint32_t tmem_holder;
    __shared__ int ok_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * g.nt;
    const int NT = g.nt;
    const uint32_t a_bytes = kBM * kBK * 2, b_bytes = (uint32_t)NT * kBK * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    const uint32_t tmem_cols = g.tmem_cols;
    // split-K: this CTA sums K range [kb, ke) (whole 64-wide slices: kchunk is a multiple of
    // kBK) into its own partial; a second kernel adds the partials in a fixed order
    const int kb = g.kchunk > 0 ? zsplit * g.kchunk : 0;
    const int ke = g.kchunk > 0 ? min(g.K, kb + g.kchunk) : g.K;
    const int nk = (ke - kb + kBK - 1) / kBK;
    const int ns = g.stages;              // ring stages in use (1..kStages), set by the launcher

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
        ok_flag = 1;
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

    if (tid == 0) {
        const uint32_t idesc = idesc_bf16(kBM, NT);
        const uint32_t base = smem_u32(smem);
        auto load_slice = [&](int kt) {
            const int st = kt % ns;
            const uint32_t sa = base + st * stage_bytes, sb = sa + a_bytes;
            mbar_expect_tx(&full[st], stage_bytes);
            const int k0 = kb + kt * kBK;
#pragma unroll
            for (int kg = 0; kg < kBK / 8; ++kg) {
                tma_load_2d(sa + kg * (kBM * 16), &mapA, k0 + 8 * kg, m0, &full[st]);
                tma_load_2d(sb + kg * (NT * 16), &mapB, k0 + 8 * kg, n0, &full[st]);
            }
        };
        bool good = true;
        int committed = 0;              // slices whose MMAs were committed
        const int pre = nk < ns ? nk : ns;
        for (int kt = 0; kt < pre; ++kt) load_slice(kt);
        for (int kt = 0; kt < nk && good; ++kt) {
            const int st = kt % ns;
            const uint32_t par = (uint32_t)(kt / ns) & 1u;
            if (!mbar_wait(&full[st], par)) { good = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = base + st * stage_bytes, b0 = a0 + a_bytes;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
                const uint64_t ad = sdesc(a0 + kk * 2 * (kBM * 16), kBM * 16, 128);
                const uint64_t bd = sdesc(b0 + kk * 2 * (NT * 16), NT * 16, 128);
                mma_bf16(tmem, ad, bd, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&empty[st]);
            committed = kt + 1;
            if (kt + ns < nk) {
                // the stage is refilled once its MMAs have read it
                if (!mbar_wait(&empty[st], par)) { good = false; break; }
                load_slice(kt + ns);
            }
        }
        // the last commit covers every MMA; wait for it (bounded)
        if (good && committed > 0)
            good = mbar_wait(&empty[(committed - 1) % ns], (uint32_t)((committed - 1) / ns) & 1u);
        if (!good) {
            if (g.err) atomicOr(g.err, 2);
            // bounded chance for copies and MMAs still in flight to finish
            for (int i = 0; i < ns; ++i) (void)mbar_wait(&empty[i], 0);
            ok_flag = 0;
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok_flag) {
        if (g.kchunk > 0) {
            GemmArgs gp = g;
            gp.C = g.part + (long)zsplit * g.M * g.N;
            gp.ldc = g.N;
            gp.Cb = nullptr;
            epilogue(gp, tmem, m0, n0, NT, nk > 0);
        } else {
            epilogue(g, tmem, m0, n0, NT, nk > 0);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

__global__ void __launch_bounds__(kGemmThreads) k_gemm_bf16_tma(const __grid_constant__ CUtensorMap mapA,
                                                                const __grid_constant__ CUtensorMap mapB, GemmArgs g)
{
    gemm_tma_body(&mapA, &mapB, g, (int)blockIdx.z);
}

// The same GEMM for the members of an ensemble, one launch: blockIdx.z = member x S + split.
__global__ void __launch_bounds__(kGemmThreads) k_gemm_bf16_tma_group(const __grid_constant__ GroupGemm G)
{
    const int member = (int)blockIdx.z / G.S, split = (int)blockIdx.z - member * G.S;
    gemm_tma_body(&G.ma[member], &G.mb[member], G.g[member], split);
}

// ---------------------------------------------------------------------------------------
// Shapes of the whole-network inference kernel below: hidden width 256, outputs padded to
// 80, an activation tile of 128 x 256 BF16, a weight slice of 256 rows x 64 K.
// ---------------------------------------------------------------------------------------
constexpr int kFusedHid = 256;
constexpr int kFusedOutPad = 80;      // 66 outputs padded to a multiple of 16
constexpr uint32_t kHBytes = kBM * kFusedHid * 2;          // 65536
constexpr uint32_t kWStageBytes = kFusedHid * kBK * 2;     // 32768

// core-matrix offset of (row r, 8-column group kg) in a K-major tile of `rows` rows
__device__ __forceinline__ uint32_t cm_off(int r, int kg, int rows) { return kg * (rows * 16) + (r >> 3) * 128 + (r & 7) * 16; }

// ---------------------------------------------------------------------------------------
// The inference pass, persistent and warp-specialised: one CTA per SM takes 128-sample
// tiles two at a time and alternates them, so that the tensor cores work on one tile while
// the epilogue warps work on the other.  Per tile x (0, 1): an activation buffer H_x (BF16,
// canonical K-major, 64 KB) and a 256-column accumulator in tensor memory (both tiles: all
// 512 columns).  Warp 0 streams the weight slices (64-wide K slices, 256 rows x 128 bytes)
// with TMA into a 2-stage ring, 128-byte swizzled; warp 1 issues the MMAs of job (x, layer)
// once H_x holds that layer's input and frees each ring stage by tcgen05.commit; warps
// 2-17 run the epilogue of job (x, layer) when its accumulator is complete: gelu(Z + b) as
// BF16 back into H_x (the next layer's input), or Y for the output layer followed by the
// inputs of the tile's successor.  Jobs run in the order (pair, layer, tile) in every role.
// mbarriers: ring stage full / empty, accumulator x complete, H_x ready (16 epilogue warps).
// Every wait is bounded; a wait that runs out raises a shared abort flag that ends every
// role's loop, after which the CTA waits (bounded) for its own copies and MMAs, frees its
// tensor memory and returns.
// ---------------------------------------------------------------------------------------
constexpr int kPPThreads = 18 * 32;
constexpr uint32_t kW1Bytes = kFusedHid * 16 * 2;          // layer-1 weights, K padded to 16
constexpr int kPPStages = 2;

size_t pp_smem_bytes() { return 2 * (size_t)kHBytes + kPPStages * (size_t)kWStageBytes + kW1Bytes + 1024; }

// descriptor of a K-major operand in the 128-byte swizzled layout: rows of 128 bytes, 8-row
// groups 1024 bytes apart (stride-dimension offset), swizzle mode 2 at bits 61-63; the
// leading-dimension offset is unused for K extents within one 128-byte row
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// bounded wait of a thread that has nothing else to do: it backs off between polls so
// that the warps doing arithmetic on its SM sub-partition keep the issue slots
__device__ __forceinline__ bool mbar_wait_idle(uint64_t* bar, uint32_t parity)
{
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > kWaitNs) return false;
        __nanosleep(64);
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct PPArgs {
    int B, ntiles, npairs;
    const __nv_bfloat16* X;
    int ld_x;
    const __nv_bfloat16* W1;
    const float* bias[5];
    float* Y;
    int* err;
};

__global__ void __launch_bounds__(kPPThreads, 1) k_mlp_forward_pp(const __grid_constant__ CUtensorMap mW2,
                                                                 const __grid_constant__ CUtensorMap mW3,
                                                                 const __grid_constant__ CUtensorMap mW4,
                                                                 const __grid_constant__ CUtensorMap mW5,
                                                                 PPArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* Hbuf = smem;                                   // H_0, H_1
    unsigned char* Wring = smem + 2 * kHBytes;                    // 2 stages, 1024-aligned
    unsigned char* W1s = Wring + kPPStages * kWStageBytes;        // layer-1 weights
    __shared__ __align__(16) float sbias[4 * kFusedHid + kFusedOutPad];
    __shared__ uint64_t wfull[kPPStages], wempty[kPPStages], accfull[2], hready[2];
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    if (tid == 0) {
        for (int k = 0; k < kPPStages; ++k) { mbar_init(&wfull[k], 1); mbar_init(&wempty[k], 1); }
        for (int x = 0; x < 2; ++x) { mbar_init(&accfull[x], 1); mbar_init(&hready[x], 16); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int k = tid; k < 4 * kFusedHid + kFusedOutPad; k += kPPThreads) {
        const int l = k / kFusedHid, n = k - l * kFusedHid;
        sbias[k] = l < 4 ? a.bias[l][n] : (n < SALEC_MLP_OUT_N ? a.bias[4][n] : 0.0f);
    }
    for (int n = tid; n < kFusedHid; n += kPPThreads) {
        *reinterpret_cast<uint4*>(W1s + cm_off(n, 0, kFusedHid)) = *reinterpret_cast<const uint4*>(a.W1 + (long)n * a.ld_x);
        *reinterpret_cast<uint4*>(W1s + cm_off(n, 1, kFusedHid)) = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;
    // tile of slot x of the k-th pair of this CTA (-1: none)
    auto tile_of = [&](int k, int x) {
        const int t = 2 * (blockIdx.x + k * G) + x;
        return (blockIdx.x + k * G < a.npairs && t < a.ntiles) ? t : -1;
    };
    const int npairs_mine = a.npairs > (int)blockIdx.x ? (a.npairs - 1 - (int)blockIdx.x) / G + 1 : 0;

    if (warp == 0) {
        // ---- weight producer ----
        if (lane == 0) {
            int fills[kPPStages] = {0, 0};
            int stage = 0;
            for (int k = 0; k < npairs_mine && !abort_flag; ++k)
                for (int l = 1; l < 5 && !abort_flag; ++l)
                    for (int x = 0; x < 2 && !abort_flag; ++x) {
                        if (tile_of(k, x) < 0) continue;
                        const int N = l == 4 ? kFusedOutPad : kFusedHid;
                        const CUtensorMap* map = l == 1 ? &mW2 : l == 2 ? &mW3 : l == 3 ? &mW4 : &mW5;
                        for (int kt = 0; kt < kFusedHid / kBK; ++kt) {
                            if (fills[stage] > 0 && !mbar_wait_idle(&wempty[stage], (uint32_t)(fills[stage] - 1) & 1u)) {
                                abort_flag = 1;
                                break;
                            }
                            mbar_expect_tx(&wfull[stage], (uint32_t)N * 128u);
                            tma_load_2d(smem_u32(Wring + stage * kWStageBytes), map, kt * kBK, 0, &wfull[stage]);
                            ++fills[stage];
                            stage ^= 1;
                        }
                    }
            // the last copies of each stage land before the CTA's memory can go away
            for (int st = 0; st < kPPStages; ++st)
                if (fills[st] > 0) (void)mbar_wait(&wfull[st], (uint32_t)(fills[st] - 1) & 1u);
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            int used[kPPStages] = {0, 0}, hwait[2] = {0, 0}, commits[2] = {0, 0};
            int stage = 0;
            const uint32_t w1 = smem_u32(W1s);
            for (int k = 0; k < npairs_mine && !abort_flag; ++k)
                for (int l = 0; l < 5 && !abort_flag; ++l)
                    for (int x = 0; x < 2 && !abort_flag; ++x) {
                        if (tile_of(k, x) < 0) continue;
                        if (!mbar_wait_idle(&hready[x], (uint32_t)(hwait[x]++) & 1u)) { abort_flag = 1; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const int N = l == 4 ? kFusedOutPad : kFusedHid;
                        const uint32_t idesc = idesc_bf16(kBM, N);
                        const uint32_t acc = tmem + (uint32_t)(x * kFusedHid);
                        const uint32_t hb = smem_u32(Hbuf + x * kHBytes);
                        if (l == 0) {
                            mma_bf16(acc, sdesc(hb, kBM * 16, 128), sdesc(w1, kFusedHid * 16, 128), idesc, 0u);
                        } else {
                            for (int kt = 0; kt < kFusedHid / kBK; ++kt) {
                                if (!mbar_wait(&wfull[stage], (uint32_t)(used[stage]++) & 1u)) { abort_flag = 1; break; }
                                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                                const uint32_t wb = smem_u32(Wring + stage * kWStageBytes);
#pragma unroll
                                for (int kk = 0; kk < kBK / 16; ++kk) {
                                    const uint64_t ad = sdesc(hb + (kt * (kBK / 8) + 2 * kk) * (kBM * 16), kBM * 16, 128);
                                    mma_bf16(acc, ad, sdesc_sw128(wb + kk * 32), idesc, (kt > 0 || kk > 0) ? 1u : 0u);
                                }
                                mma_commit(&wempty[stage]);
                                stage ^= 1;
                            }
                            if (abort_flag) break;
                        }
                        mma_commit(&accfull[x]);
                        ++commits[x];
                    }
            // MMAs still in flight finish before the tensor memory is freed
            if (abort_flag)
                for (int x = 0; x < 2; ++x)
                    if (commits[x] > 0) (void)mbar_wait(&accfull[x], (uint32_t)(commits[x] - 1) & 1u);
        }
    } else {
        // ---- epilogue: warps 2-17; lane quarter q (TMEM lanes 32q..), column quarter cq ----
        const int q = warp & 3, cq = (warp - 2) >> 2;
        const int r = q * 32 + lane;                         // row of the tile
        const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
        int accw[2] = {0, 0};
        // the warp decides together: an abort seen by any lane ends the warp's loop
        auto aborted = [&]() { return __any_sync(0xffffffffu, abort_flag != 0); };
        // inputs of tile t into H_x: X rows (8 BF16 = one core-matrix row), K padded to 16
        auto stage_inputs = [&](int x, int t) {
            if (cq == 0) {
                const int m = t * kBM + r;
                uint4 xv = make_uint4(0u, 0u, 0u, 0u);
                if (m < a.B) xv = *reinterpret_cast<const uint4*>(a.X + (long)m * a.ld_x);
                unsigned char* H = Hbuf + x * kHBytes;
                *reinterpret_cast<uint4*>(H + cm_off(r, 0, kBM)) = xv;
                *reinterpret_cast<uint4*>(H + cm_off(r, 1, kBM)) = make_uint4(0u, 0u, 0u, 0u);
            }
        };
        auto release = [&](int x) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&hready[x]);
        };
        for (int x = 0; x < 2; ++x) {
            const int t = tile_of(0, x);
            if (t < 0) continue;
            stage_inputs(x, t);
            release(x);
        }
        bool stop = aborted();
        for (int k = 0; k < npairs_mine && !stop; ++k)
            for (int l = 0; l < 5 && !stop; ++l)
                for (int x = 0; x < 2 && !(stop = aborted()); ++x) {
                    const int t = tile_of(k, x);
                    if (t < 0) continue;
                    const bool ok = __all_sync(0xffffffffu, mbar_wait(&accfull[x], (uint32_t)(accw[x]++) & 1u));
                    if (!ok) {
                        abort_flag = 1;
                        stop = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t tacc = trow + (uint32_t)(x * kFusedHid);
                    const int m = t * kBM + r;
                    const bool live = m < a.B;
                    const float* bias = sbias + l * kFusedHid;
                    if (l < 4) {
                        unsigned char* H = Hbuf + x * kHBytes;
#pragma unroll 1
                        for (int c0 = cq * 64; c0 < cq * 64 + 64; c0 += 16) {
                            float v[16];
                            tmem_ld16(tacc + (uint32_t)c0, v);
                            uint32_t w[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
                            if (live) {
                                const float4* b4 = reinterpret_cast<const float4*>(bias + c0);
#pragma unroll
                                for (int qq = 0; qq < 4; ++qq) {
                                    const float4 b = b4[qq];
                                    const f32x2 glo = gelu_pair(f2add(f2(v[4 * qq], v[4 * qq + 1]), f2(b.x, b.y)));
                                    const f32x2 ghi = gelu_pair(f2add(f2(v[4 * qq + 2], v[4 * qq + 3]), f2(b.z, b.w)));
                                    const __nv_bfloat162 lo = __floats2bfloat162_rn(f2lo(glo), f2hi(glo));
                                    const __nv_bfloat162 hi = __floats2bfloat162_rn(f2lo(ghi), f2hi(ghi));
                                    w[2 * qq] = *reinterpret_cast<const uint32_t*>(&lo);
                                    w[2 * qq + 1] = *reinterpret_cast<const uint32_t*>(&hi);
                                }
                            }
                            *reinterpret_cast<uint4*>(H + cm_off(r, (c0 >> 3), kBM)) = make_uint4(w[0], w[1], w[2], w[3]);
                            *reinterpret_cast<uint4*>(H + cm_off(r, (c0 >> 3) + 1, kBM)) = make_uint4(w[4], w[5], w[6], w[7]);
                        }
                        release(x);
                    } else {
                        for (int c0 = cq * 16; c0 < kFusedOutPad; c0 += 64) {
                            float v[16];
                            tmem_ld16(tacc + (uint32_t)c0, v);
                            if (live) {
                                float* y = a.Y + (long)m * SALEC_MLP_OUT_N + c0;
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    if (c0 + j < SALEC_MLP_OUT_N) y[j] = v[j] + bias[c0 + j];
                            }
                        }
                        // the accumulator is read and H_x is free: the successor's inputs
                        const int tn = tile_of(k + 1, x);
                        if (tn >= 0) {
                            stage_inputs(x, tn);
                            release(x);
                        }
                    }
                }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_flag && tid == 0 && a.err) atomicOr(a.err, 4);
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// Column sums of a BF16 matrix (bias gradients): out[n] = sum_m G[m][n].
// Column sums in two passes (many rows, few columns): block (x, y) sums rows y, y + Y, ...
// of its columns into part[y][n]; the second pass adds the Y partials in order.
// split-K partials [S][M][N] into C (row stride ldc), in split order; with Cb, column N - 1
// goes to Cb[m] and C holds the other columns
__global__ void k_splitk_reduce(const float* __restrict__ part, int S, int M, int N, float* __restrict__ C, long ldc,
                                float* __restrict__ Cb)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long)M * N) return;
    float s = 0.0f;
    for (int p = 0; p < S; ++p) s += part[(long)p * M * N + k];
    const long m = k / N;
    const int n = (int)(k - m * N);
    if (Cb && n == N - 1)
        Cb[m] = s;
    else
        C[m * ldc + n] = s;
}

// The split-K reduction of a group's GEMMs: blockIdx.y = member.
struct GroupReduce {
    const float* part[kMaxGroup];
    float* C[kMaxGroup];
    float* Cb[kMaxGroup];
    long ldc;
    int S, M, N;
};
__global__ void k_splitk_reduce_group(const __grid_constant__ GroupReduce R)
{
    const int g = blockIdx.y;
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long)R.M * R.N) return;
    const float* part = R.part[g];
    float s = 0.0f;
    for (int p = 0; p < R.S; ++p) s += part[(long)p * R.M * R.N + k];
    const long m = k / R.N;
    const int n = (int)(k - m * R.N);
    if (R.Cb[g] && n == R.N - 1)
        R.Cb[g][m] = s;
    else
        R.C[g][m * R.ldc + n] = s;
}

// FP32 -> BF16 inputs of the first layer: rows of `cols` values into rows of `ld`, the
// padding zero.
__global__ void k_inputs_bf16(const float* __restrict__ x, int rows, int cols, int ld, __nv_bfloat16* __restrict__ y,
                              __nv_bfloat16* __restrict__ yT, long ldT)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)rows * ld) return;
    const long r = i / ld;
    const int c = (int)(i - r * ld);
    const __nv_bfloat16 v = __float2bfloat16_rn(c < cols ? x[r * cols + c] : 0.0f);
    y[i] = v;
    if (yT && c < cols) yT[(long)c * ldT + r] = v;
}

// Adam on the FP32 master parameters; refreshes the BF16 copy of every weight.  wmap[i] is
// the index of parameter i in the BF16 weight block, or -1 for a bias.
__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m1, float* __restrict__ m2,
                       const float* __restrict__ grad, long n, AdamArgs a, const int* __restrict__ wmap,
                       __nv_bfloat16* __restrict__ wbf, const int* __restrict__ wmapT, __nv_bfloat16* __restrict__ wbfT)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float lr = a.lr, c1 = a.c1, c2 = a.c2;
    if (a.ts) {
        lr = a.ts->lr;
        c1 = a.ts->c1;
        c2 = a.ts->c2;
    }
    const float g = grad[i];
    const float mi = a.beta1 * m1[i] + (1.0f - a.beta1) * g;
    const float vi = a.beta2 * m2[i] + (1.0f - a.beta2) * g * g;
    m1[i] = mi;
    m2[i] = vi;
    const float th = theta[i] - lr * (mi * c1) / (sqrtf(vi * c2) + a.eps);
    theta[i] = th;
    const int w = wmap[i];
    if (w >= 0) wbf[w] = __float2bfloat16_rn(th);
    if (wmapT) {
        const int wt = wmapT[i];
        if (wt >= 0) wbfT[wt] = __float2bfloat16_rn(th);
    }
}

__global__ void k_train_reset(TrainState* ts, int t0)
{
    ts->k = 0;
    ts->t0 = t0;
}

// The step's learning rate and Adam bias corrections (the same double-precision formula the
// single-step call evaluates on the host), and the loss accumulator zeroed.
__global__ void k_train_begin(TrainState* ts, const float* __restrict__ lr_dev, float beta1, float beta2, double* loss)
{
    const int k = ts->k + 1;
    const double t = (double)(ts->t0 + k);
    ts->k = k;
    ts->lr = lr_dev[k - 1];
    ts->c1 = (float)(1.0 / (1.0 - pow((double)beta1, t)));
    ts->c2 = (float)(1.0 / (1.0 - pow((double)beta2, t)));
    *loss = 0.0;
}

// Adam for the members of a group (blockIdx.y = member): the arithmetic of k_adam.
__global__ void k_adam_group(const __grid_constant__ AdamGroup A, long n, float beta1, float beta2, float eps,
                             const int* __restrict__ wmap, const int* __restrict__ wmapT)
{
    const int g = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const TrainState* ts = A.ts[g];
    const float lr = ts->lr, c1 = ts->c1, c2 = ts->c2;
    float* m1 = A.m1[g];
    float* m2 = A.m2[g];
    const float gr = A.grad[g][i];
    const float mi = beta1 * m1[i] + (1.0f - beta1) * gr;
    const float vi = beta2 * m2[i] + (1.0f - beta2) * gr * gr;
    m1[i] = mi;
    m2[i] = vi;
    const float th = A.theta[g][i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    A.theta[g][i] = th;
    const int w = wmap[i];
    if (w >= 0) A.wbf[g][w] = __float2bfloat16_rn(th);
    const int wt = wmapT[i];
    if (wt >= 0) A.wbfT[g][wt] = __float2bfloat16_rn(th);
}

// k_train_begin for every member of a group (thread = member).
__global__ void k_train_begin_group(const __grid_constant__ BeginGroup B, int n, const float* __restrict__ lr_dev,
                                    float beta1, float beta2)
{
    const int g = threadIdx.x;
    if (g >= n) return;
    TrainState* ts = B.ts[g];
    const int k = ts->k + 1;
    const double t = (double)(ts->t0 + k);
    ts->k = k;
    ts->lr = lr_dev[k - 1];
    ts->c1 = (float)(1.0 / (1.0 - pow((double)beta1, t)));
    ts->c2 = (float)(1.0 / (1.0 - pow((double)beta2, t)));
    *B.loss[g] = 0.0;
}

// BF16 copy of the weights from the FP32 parameters.
__global__ void k_refresh_bf16(const float* __restrict__ theta, long n, const int* __restrict__ wmap,
                               __nv_bfloat16* __restrict__ wbf, const int* __restrict__ wmapT,
                               __nv_bfloat16* __restrict__ wbfT)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int w = wmap[i];
    if (w >= 0) wbf[w] = __float2bfloat16_rn(theta[i]);
    if (wmapT) {
        const int wt = wmapT[i];
        if (wt >= 0) wbfT[wt] = __float2bfloat16_rn(theta[i]);
    }
}

size_t gemm_smem_bytes(int nt) { return 2 * (size_t)(kBM * kBK * 2 + nt * kBK * 2) + 1024; }

namespace {

// cuTensorMapEncodeTiled from the driver (looked up once, shared with the solver's copy kernel)
TmaEncodeTiledFn encode_tiled() { return tma_encode_tiled(); }

// 2-D map of a row-major BF16 matrix [rows][K] with row stride ld elements; boxes of 8
// elements (16 bytes) x box_rows rows.  False when TMA cannot address it (alignment).
bool make_map(CUtensorMap* map, const void* base, long rows, long K, long ld, int box_rows)
{
    const TmaEncodeTiledFn fn = encode_tiled();
    if (!fn || rows < 1 || K < 1 || (reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {8u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tma_smem_bytes(int nt, int stages = kStages) { return (size_t)stages * (kBM * kBK * 2 + nt * kBK * 2) + 1024; }

// The same matrix as 64-element (128-byte) x box_rows boxes in the 128-byte swizzled
// layout (one box is one K slice of box_rows rows).
bool make_map_sw128(CUtensorMap* map, const void* base, long rows, long K, long ld, int box_rows)
{
    const TmaEncodeTiledFn fn = encode_tiled();
    if (!fn || rows < 1 || K < 64 || (reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// SM count and the TMA kernels' shared-memory attribute, per device (set once)
cudaError_t tma_device_setup(int dev, int* sms)
{
    static int sm_count[64] = {};
    static bool attr_tma[64] = {};
    cudaError_t e = cudaSuccess;
    if (!sm_count[dev]) {
        e = cudaDeviceGetAttribute(&sm_count[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    if (!attr_tma[dev]) {
        e = cudaFuncSetAttribute(k_gemm_bf16_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes(kMaxNT_TMA));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_gemm_bf16_tma_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tma_smem_bytes(kMaxNT_TMA));
        if (e != cudaSuccess) return e;
        attr_tma[dev] = true;
    }
    *sms = sm_count[dev];
    return cudaSuccess;
}

// The TMA-fed kernel's plan for one product: tile width, K split, ring stages, tensor-memory
// columns (into g), and the grid (mt row tiles, ntl column tiles, S splits).
void plan_tma(GemmArgs& g, int sms, int* mt_out, int* ntl_out, int* S_out)
{
    const int mt = (g.M + kBM - 1) / kBM;
    auto round16 = [](int x) { return (x + 15) / 16 * 16; };
    auto tiles_n = [&](int w) { return (g.N + w - 1) / w; };
    // a long K over few output tiles (the weight gradients, K = batch): wide tiles and K
    // split over up to kMaxSplit CTAs per tile, each storing a partial
    int ntn = tiles_n(kMaxNT_TMA);
    int nt = round16((g.N + ntn - 1) / ntn);
    int S = 1;
    g.kchunk = 0;
    if (g.epi == kEpiStore && !g.bias && g.part && g.K >= 4 * kBK && mt * ntn < sms / 2) {
        const int slices = (g.K + kBK - 1) / kBK;
        S = (sms + mt * ntn - 1) / (mt * ntn);
        S = S < kMaxSplit ? S : kMaxSplit;
        S = S < (slices + 1) / 2 ? S : (slices + 1) / 2;          // at least 2 slices each
        if (S > 1) {
            g.kchunk = (slices + S - 1) / S * kBK;
            S = (g.K + g.kchunk - 1) / g.kchunk;
        } else {
            S = 1;
        }
    } else {
        // otherwise narrower tiles (down to 32 columns) until the tiles fill the SMs:
        // the epilogue of a tile is the longest part of a CTA, and it shrinks with it
        while (mt * tiles_n(nt) < sms && nt > 32) {
            ntn *= 2;
            const int w = round16((g.N + ntn - 1) / ntn);
            nt = w > 32 ? w : 32;
        }
    }
    g.nt = nt;
    int cols = 32;
    while (cols < nt) cols <<= 1;
    g.tmem_cols = cols;
    // narrow tiles keep two stages in flight: 41 KB of shared memory, five CTAs per SM, so
    // that concurrent GEMMs (ensemble members) overlap
    g.stages = nt <= 64 ? 2 : kStages;
    *mt_out = mt;
    *ntl_out = tiles_n(nt);
    *S_out = S;
}

cudaError_t launch_gemm(const GemmArgs& g0, cudaStream_t s)
{
    GemmArgs g = g0;
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    // both operands K-major with 16-byte rows: the TMA-fed kernel
    if (g.K > 0 && g.a_sk == 1 && g.b_sk == 1) {
        int sms = 0, mt = 0, ntl = 0, S = 1;
        e = tma_device_setup(dev, &sms);
        if (e != cudaSuccess) return e;
        plan_tma(g, sms, &mt, &ntl, &S);
        CUtensorMap ma, mb;
        if (make_map(&ma, g.A, g.M, g.K, g.a_sm, kBM) && make_map(&mb, g.B, g.N, g.K, g.b_sn, g.nt)) {
            dim3 grid((unsigned)mt, (unsigned)ntl, (unsigned)S);
            k_gemm_bf16_tma<<<grid, kGemmThreads, tma_smem_bytes(g.nt, g.stages), s>>>(ma, mb, g);
            e = cudaGetLastError();
            if (e != cudaSuccess || g.kchunk == 0) return e;
            const long mn = (long)g.M * g.N;
            k_splitk_reduce<<<(unsigned)((mn + 255) / 256), 256, 0, s>>>(g.part, S, g.M, g.N, g.C, g.ldc, g.Cb);
            return cudaGetLastError();
        }
        g.kchunk = 0;
    }
    const int nt = ((g.N < kMaxNT ? g.N : kMaxNT) + 15) / 16 * 16;
    g.nt = nt;
    int cols = 32;
    while (cols < nt) cols <<= 1;
    g.tmem_cols = cols;
    const size_t smem = gemm_smem_bytes(nt);
    // few output tiles and a long K (the weight gradients: K = batch): split K over up to
    // kMaxSplit CTAs per tile, each summing a range of 64-multiples into a partial
    const int tiles = ((g.M + kBM - 1) / kBM) * ((g.N + nt - 1) / nt);
    int S = 1;
    g.kchunk = 0;
    if (g.epi == kEpiStore && !g.bias && g.part && tiles < 64 && g.K >= 4 * kBK) {
        S = (g.K + 2 * kBK - 1) / (2 * kBK);                      // at least 2 slices each
        const int want = (128 + tiles - 1) / tiles;
        S = S < want ? S : want;
        S = S < kMaxSplit ? S : kMaxSplit;
        if (S > 1) {
            const int slices = (g.K + kBK - 1) / kBK;
            g.kchunk = (slices + S - 1) / S * kBK;
            S = (g.K + g.kchunk - 1) / g.kchunk;
        } else {
            S = 1;
        }
    }
    // the attribute is per device
    static bool attr_set[64] = {};
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem_bytes(kMaxNT));
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    dim3 grid((unsigned)((g.M + kBM - 1) / kBM), (unsigned)((g.N + nt - 1) / nt), (unsigned)S);
    k_gemm_bf16<<<grid, kGemmThreads, smem, s>>>(g);
    e = cudaGetLastError();
    if (e != cudaSuccess || g.kchunk == 0) return e;
    const long mn = (long)g.M * g.N;
    k_splitk_reduce<<<(unsigned)((mn + 255) / 256), 256, 0, s>>>(g.part, S, g.M, g.N, g.C, g.ldc, g.Cb);
    return cudaGetLastError();
}

cudaError_t launch_gemm_group(const GemmArgs* g0, int n, cudaStream_t s)
{
    if (n < 1 || n > kMaxGroup) return cudaErrorInvalidValue;
    const GemmArgs& a = g0[0];
    if (a.M <= 0 || a.N <= 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    bool tma = a.K > 0 && a.a_sk == 1 && a.b_sk == 1;
    GroupGemm G;
    int mt = 0, ntl = 0, S = 1;
    if (tma) {
        int sms = 0;
        e = tma_device_setup(dev, &sms);
        if (e != cudaSuccess) return e;
        for (int k = 0; k < n && tma; ++k) {
            G.g[k] = g0[k];
            plan_tma(G.g[k], sms, &mt, &ntl, &S);      // the same plan as a member launched alone
            tma = make_map(&G.ma[k], G.g[k].A, G.g[k].M, G.g[k].K, G.g[k].a_sm, kBM) &&
                  make_map(&G.mb[k], G.g[k].B, G.g[k].N, G.g[k].K, G.g[k].b_sn, G.g[k].nt);
        }
    }
    if (!tma) {
        // operands the TMA cannot address: each member on its own
        for (int k = 0; k < n; ++k)
            if ((e = launch_gemm(g0[k], s)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    G.n = n;
    G.S = S;
    const GemmArgs& p = G.g[0];
    dim3 grid((unsigned)mt, (unsigned)ntl, (unsigned)(S * n));
    k_gemm_bf16_tma_group<<<grid, kGemmThreads, tma_smem_bytes(p.nt, p.stages), s>>>(G);
    e = cudaGetLastError();
    if (e != cudaSuccess || p.kchunk == 0) return e;
    GroupReduce R;
    for (int k = 0; k < n; ++k) {
        R.part[k] = G.g[k].part;
        R.C[k] = G.g[k].C;
        R.Cb[k] = G.g[k].Cb;
    }
    R.ldc = p.ldc;
    R.S = S;
    R.M = p.M;
    R.N = p.N;
    const long mn = (long)p.M * p.N;
    k_splitk_reduce_group<<<dim3((unsigned)((mn + 255) / 256), (unsigned)n), 256, 0, s>>>(R);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward_fused(const FusedLaunch& f, cudaStream_t s)
{
    if (f.B <= 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        // persistent ping-pong kernel: one CTA per SM, pairs of 128-sample tiles
        CUtensorMap m2, m3, m4, m5;
        if (!make_map_sw128(&m2, f.W[1], kFusedHid, kFusedHid, kFusedHid, kFusedHid) ||
            !make_map_sw128(&m3, f.W[2], kFusedHid, kFusedHid, kFusedHid, kFusedHid) ||
            !make_map_sw128(&m4, f.W[3], kFusedHid, kFusedHid, kFusedHid, kFusedHid) ||
            !make_map_sw128(&m5, f.W[4], SALEC_MLP_OUT_N, kFusedHid, kFusedHid, kFusedOutPad))
            return cudaErrorNotSupported;
        static bool attr_pp[64] = {};
        static int nsm[64] = {};
        if (!attr_pp[dev]) {
            e = cudaFuncSetAttribute(k_mlp_forward_pp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pp_smem_bytes());
            if (e != cudaSuccess) return e;
            e = cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            attr_pp[dev] = true;
        }
        PPArgs a;
        a.B = f.B;
        a.ntiles = (f.B + kBM - 1) / kBM;
        a.npairs = (a.ntiles + 1) / 2;
        a.X = f.X; a.ld_x = f.ld_x; a.W1 = f.W[0];
        for (int l = 0; l < 5; ++l) a.bias[l] = f.bias[l];
        a.Y = f.Y; a.err = f.err;
        const int grid = a.npairs < nsm[dev] ? a.npairs : nsm[dev];
        k_mlp_forward_pp<<<(unsigned)grid, kPPThreads, pp_smem_bytes(), s>>>(m2, m3, m4, m5, a);
        return cudaGetLastError();
    }
}

cudaError_t launch_inputs_bf16(const float* x, int rows, int cols, int ld, __nv_bfloat16* y, cudaStream_t s,
                               __nv_bfloat16* yT, long ldT)
{
    const long n = (long)rows * ld;
    if (n <= 0) return cudaSuccess;
    k_inputs_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, rows, cols, ld, y, yT, ldT);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, float* m1, float* m2, const float* grad, long n, const AdamArgs& a,
                        const int* wmap, __nv_bfloat16* wbf, cudaStream_t s, const int* wmapT, __nv_bfloat16* wbfT)
{
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(theta, m1, m2, grad, n, a, wmap, wbf, wmapT, wbfT);
    return cudaGetLastError();
}

cudaError_t launch_train_reset(TrainState* ts, int t0, cudaStream_t s)
{
    k_train_reset<<<1, 1, 0, s>>>(ts, t0);
    return cudaGetLastError();
}

cudaError_t launch_train_begin(TrainState* ts, const float* lr_dev, float beta1, float beta2, double* loss, cudaStream_t s)
{
    k_train_begin<<<1, 1, 0, s>>>(ts, lr_dev, beta1, beta2, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam_group(const AdamGroup& a, int n, long np, float beta1, float beta2, float eps, const int* wmap,
                              const int* wmapT, cudaStream_t s)
{
    if (n < 1 || n > kMaxGroup) return cudaErrorInvalidValue;
    k_adam_group<<<dim3((unsigned)((np + 255) / 256), (unsigned)n), 256, 0, s>>>(a, np, beta1, beta2, eps, wmap, wmapT);
    return cudaGetLastError();
}

cudaError_t launch_train_begin_group(const BeginGroup& b, int n, const float* lr_dev, float beta1, float beta2,
                                     cudaStream_t s)
{
    if (n < 1 || n > kMaxGroup) return cudaErrorInvalidValue;
    k_train_begin_group<<<1, 32, 0, s>>>(b, n, lr_dev, beta1, beta2);
    return cudaGetLastError();
}

cudaError_t launch_refresh_bf16(const float* theta, long n, const int* wmap, __nv_bfloat16* wbf, cudaStream_t s,
                                const int* wmapT, __nv_bfloat16* wbfT)
{
    k_refresh_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(theta, n, wmap, wbf, wmapT, wbfT);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace salec
