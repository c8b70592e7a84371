// Arithmetic issue rates of the instructions the back-projection's inner loop
// is made of, measured on the running GPU: the denominator of its roofline.
//
// The back-projection of Algorithm 4 is bound by the per-update arithmetic of
// Algorithms 3 and 4 (the projection bytes per update are tiny), so the
// roofline's peak is an arithmetic rate.  Whether the packed two-wide FP32
// FMA (fma.rn.f32x2) raises the FP32 operation rate above one FMA per lane
// and clock, and what the half2 FMA and the FP16-input FP32 FMA
// (fma.rn.f32.f16) of the 16-bit storage path deliver, is measured here
// rather than assumed.
//
// Kernel: one block of 1024 threads per SM (its shared memory keeps a second
// block off the SM), each thread running kChains
// independent dependency chains of one instruction kind, kUnroll chain steps
// per loop iteration; the block reads its own SM clock (clock64) around the
// loop, so a rate is lane operations per SM clock, independent of the clock
// frequency.  The loop counter adds ~3 instructions per kChains * kUnroll
// chain steps (under 3 %), so the rates are lower bounds.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ifdk_device.cuh"
#include "ifdk_internal.h"

namespace ifdk {
namespace {

constexpr int kChains = 8, kUnroll = 16, kRateThreads = 1024;

// One step of chain c for each kind; the chains never converge to a constant
// the compiler could see (the operands come from the kernel's arguments).
template <int KIND> struct Step;
template <> struct Step<IFDK_RATE_FFMA> {
    using V = float;
    static constexpr int LANES = 1;
    __device__ __forceinline__ static V init(float s, int c) { return s + (float)c; }
    __device__ __forceinline__ static void run(V &x, float b, float c)
    {
        asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x) : "f"(b), "f"(c));
    }
    __device__ __forceinline__ static float out(V x) { return x; }
};
template <> struct Step<IFDK_RATE_FFMA2> {
    using V = float2;
    static constexpr int LANES = 2;
    __device__ __forceinline__ static V init(float s, int c) { return make_float2(s + (float)c, s - (float)c); }
    __device__ __forceinline__ static void run(V &x, float b, float c)
    {
        x = __ffma2_rn(x, make_float2(b, b), make_float2(c, c));
    }
    __device__ __forceinline__ static float out(V x) { return x.x + x.y; }
};
template <> struct Step<IFDK_RATE_HFMA2> {
    using V = uint32_t;
    static constexpr int LANES = 2;
    __device__ __forceinline__ static V init(float s, int c)
    {
        const __half2 h = __floats2half2_rn(s * 1e-3f + 1e-4f * c, s * 1e-3f - 1e-4f * c);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    __device__ __forceinline__ static void run(V &x, float b, float c)
    {
        const __half2 hb = __float2half2_rn(b), hc = __float2half2_rn(c);
        asm volatile("fma.rn.f16x2 %0, %0, %1, %2;"
                     : "+r"(x)
                     : "r"(*reinterpret_cast<const uint32_t *>(&hb)), "r"(*reinterpret_cast<const uint32_t *>(&hc)));
    }
    __device__ __forceinline__ static float out(V x)
    {
        const __half2 h = *reinterpret_cast<const __half2 *>(&x);
        return __low2float(h) + __high2float(h);
    }
};
// FP32 accumulate of an FP16 product, d = a * b + d with a, b FP16 (the
// accumulate of the FP16-storage back-projection); the same with BF16 inputs
// (the u-lerp of the BF16-storage back-projection)
template <> struct Step<IFDK_RATE_FMA_F32_F16> {
    using V = float;
    static constexpr int LANES = 1;
    __device__ __forceinline__ static V init(float s, int c) { return s + (float)c; }
    __device__ __forceinline__ static void run(V &x, float b, float c)
    {
        const unsigned short hb = __half_as_ushort(__float2half_rn(b)), hc = __half_as_ushort(__float2half_rn(c));
        asm volatile("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(x) : "h"(hb), "h"(hc));
    }
    __device__ __forceinline__ static float out(V x) { return x; }
};
template <> struct Step<IFDK_RATE_FMA_F32_BF16> {
    using V = float;
    static constexpr int LANES = 1;
    __device__ __forceinline__ static V init(float s, int c) { return s + (float)c; }
    __device__ __forceinline__ static void run(V &x, float b, float c)
    {
        const unsigned short hb = __bfloat16_as_ushort(__float2bfloat16_rn(b));
        const unsigned short hc = __bfloat16_as_ushort(__float2bfloat16_rn(c));
        asm volatile("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(x) : "h"(hb), "h"(hc));
    }
    __device__ __forceinline__ static float out(V x) { return x; }
};
// Integer logic (lop3, three-input xor): the rate of the integer ops that widen
// BF16 values (shift, mask) where a kernel widens them
template <> struct Step<IFDK_RATE_LOP3> {
    using V = uint32_t;
    static constexpr int LANES = 1;
    __device__ __forceinline__ static V init(float s, int c) { return __float_as_uint(s) + (uint32_t)c; }
    __device__ __forceinline__ static void run(V &x, float b, float c)
    {
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x) : "r"(__float_as_uint(b)), "r"(__float_as_uint(c)));
    }
    __device__ __forceinline__ static float out(V x) { return (float)(x & 0xffffu); }
};

template <int KIND>
__global__ void __launch_bounds__(kRateThreads, 1)
    rate_kernel(long long iters, float seed, float b, float c, float *sink, long long *clk)
{
    using S = Step<KIND>;
    typename S::V x[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = S::init(seed + (float)threadIdx.x * 1e-6f, q);
    // the operands stay in registers: the compiler cannot fold them
    const float bb = b + (float)(threadIdx.x & 1) * 1e-7f, cc = c;
    __syncthreads();
    const long long t0 = clock64();
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int q = 0; q < kChains; ++q) S::run(x[q], bb, cc);
    }
    __syncthreads();
    const long long t1 = clock64();
    float acc = 0.0f;
#pragma unroll
    for (int q = 0; q < kChains; ++q) acc += S::out(x[q]);
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) {
        uint32_t smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        clk[3 * blockIdx.x] = t0;
        clk[3 * blockIdx.x + 1] = t1;
        clk[3 * blockIdx.x + 2] = smid;
    }
}

// Dynamic shared memory (unused) that keeps a second block off the SM, so that
// every block has its SM to itself.
constexpr int kRateSmem = 160 * 1024;

template <int KIND> int launch_rate(int blocks, long long iters, float *sink, long long *clk, cudaStream_t s)
{
    if (cudaFuncSetAttribute(rate_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRateSmem) !=
        cudaSuccess)
        return IFDK_ERR_CUDA;
    rate_kernel<KIND><<<blocks, kRateThreads, kRateSmem, s>>>(iters, 0.75f, 0.999f, 1e-3f, sink, clk);
    return cudaGetLastError() == cudaSuccess ? IFDK_OK : IFDK_ERR_CUDA;
}

}  // namespace
}  // namespace ifdk

extern "C" int ifdk_arith_rate(int kind, int blocks, long long iters, float *sink, long long *clocks, int64_t out[2],
                               void *stream)
{
    using namespace ifdk;
    if (!sink || !clocks || !out) return IFDK_ERR_INVALID;
    if (blocks < 1 || blocks > 65535 || iters < 1 || iters > ((long long)1 << 30)) return IFDK_ERR_INVALID;
    if (((uintptr_t)clocks & 7) || ((uintptr_t)sink & 3)) return IFDK_ERR_ALIGNMENT;
    int lanes = 0, rc = IFDK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    switch (kind) {
    case IFDK_RATE_FFMA: lanes = 1; rc = launch_rate<IFDK_RATE_FFMA>(blocks, iters, sink, clocks, s); break;
    case IFDK_RATE_FFMA2: lanes = 2; rc = launch_rate<IFDK_RATE_FFMA2>(blocks, iters, sink, clocks, s); break;
    case IFDK_RATE_HFMA2: lanes = 2; rc = launch_rate<IFDK_RATE_HFMA2>(blocks, iters, sink, clocks, s); break;
    case IFDK_RATE_FMA_F32_F16:
        lanes = 1;
        rc = launch_rate<IFDK_RATE_FMA_F32_F16>(blocks, iters, sink, clocks, s);
        break;
    case IFDK_RATE_LOP3: lanes = 1; rc = launch_rate<IFDK_RATE_LOP3>(blocks, iters, sink, clocks, s); break;
    case IFDK_RATE_FMA_F32_BF16:
        lanes = 1;
        rc = launch_rate<IFDK_RATE_FMA_F32_BF16>(blocks, iters, sink, clocks, s);
        break;
    default: return IFDK_ERR_INVALID;
    }
    // instructions per thread, and lane operations per instruction
    out[0] = iters * (long long)kUnroll * kChains;
    out[1] = lanes;
    return rc;
}
