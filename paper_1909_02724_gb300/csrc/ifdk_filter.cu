// Filtering stage (Algorithm 1 of the iFDK paper): cosine weight F_cos then
// the Ram-Lak ramp convolution of every detector row, computed as the dense
// Toeplitz product Q_row = T . (F_cos . E_row), T[n][m] = h(n - m), which is
// the exact linear (zero padded) convolution truncated to Nu outputs.
//
// FP32 SIMT kernel: a block computes 1024 consecutive outputs of kRows rows;
// the weighted rows and the taps the block needs sit in shared memory; every
// thread keeps 4 consecutive outputs x kRows rows in registers and slides a
// 4-tap window down the Toeplitz diagonal.  The cosine weight is applied when
// the rows are staged (or to the outputs, for the adjoint), and the epilogue
// casts to the storage type.
#include "ifdk_device.cuh"
#include "ifdk_internal.h"

namespace ifdk {
namespace {

constexpr int kRows = 4;          // rows per block
constexpr int kOutPerThread = 4;  // consecutive outputs per thread
constexpr int kFThreads = 256;
constexpr int kOutPerBlock = kFThreads * kOutPerThread;

template <typename TQ, bool ADJ>
__global__ void __launch_bounds__(kFThreads)
    filter_simt_kernel(const float *__restrict__ E, TQ *__restrict__ Q, const float *__restrict__ fcos,
                       const float *__restrict__ taps, int nu, int nv, long long rows)
{
    extern __shared__ float sm[];
    float *w = sm;                        // [kRows][nu] weighted input rows
    float *hs = sm + kRows * nu;          // taps window, see below
    const int n_lo = blockIdx.x * kOutPerBlock;
    const long long r0 = (long long)blockIdx.y * kRows;

    for (int r = 0; r < kRows; ++r) {
        const long long row = r0 + r;
        for (int m = threadIdx.x; m < nu; m += kFThreads) {
            float x = 0.0f;
            if (row < rows) {
                x = __ldg(E + row * nu + m);
                if (!ADJ) x *= __ldg(fcos + (row % nv) * nu + m);
            }
            w[r * nu + m] = x;
        }
    }
    // hs[t] = h(d) with d = t - 4 + n_lo - (nu - 1), for d in the range the block uses.
    const int hlen = kOutPerBlock + nu + 4;
    for (int t = threadIdx.x; t < hlen; t += kFThreads) {
        const int d = t - 4 + n_lo - (nu - 1);
        hs[t] = (d > -nu && d < nu) ? __ldg(taps + d + nu - 1) : 0.0f;
    }
    __syncthreads();

    const int n0 = n_lo + threadIdx.x * kOutPerThread;
    if (n0 >= nu) return;
    float acc[kRows][kOutPerThread];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int q = 0; q < kOutPerThread; ++q) acc[r][q] = 0.0f;
    // output n0+q at input m uses h(n0 + q - m) = hs[base + q - m]
    const int base = threadIdx.x * kOutPerThread + nu - 1 + 4;
    float h0 = hs[base], h1 = hs[base + 1], h2 = hs[base + 2], h3 = hs[base + 3];
    for (int m = 0; m < nu; ++m) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const float x = w[r * nu + m];
            acc[r][0] = fmaf(h0, x, acc[r][0]);
            acc[r][1] = fmaf(h1, x, acc[r][1]);
            acc[r][2] = fmaf(h2, x, acc[r][2]);
            acc[r][3] = fmaf(h3, x, acc[r][3]);
        }
        h3 = h2;
        h2 = h1;
        h1 = h0;
        h0 = hs[base - m - 1];
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const long long row = r0 + r;
        if (row >= rows) break;
#pragma unroll
        for (int q = 0; q < kOutPerThread; ++q) {
            const int n = n0 + q;
            if (n < nu) {
                float y = acc[r][q];
                if (ADJ) y *= __ldg(fcos + (row % nv) * nu + n);
                Q[row * nu + n] = Storage<TQ>::from_float(y);
            }
        }
    }
}

template <typename TQ, bool ADJ>
int launch_simt(ifdk_plan_s *p, const float *E, void *Q, cudaStream_t stream)
{
    const ifdk_geometry &g = p->g;
    const long long rows = (long long)g.np * g.nv;
    const size_t smem = sizeof(float) * ((size_t)kRows * g.nu + kOutPerBlock + g.nu + 4);
    if (smem > 220 * 1024) return IFDK_ERR_UNSUPPORTED;
    // grid.y is limited to 65535 blocks: launch whole views at a time so that
    // every launch starts on detector row 0 (the F_cos row is row % nv).
    const long long max_rows = 65535LL * kRows;
    const long long chunk = (max_rows / g.nv) * (long long)g.nv;
    if (chunk == 0) return IFDK_ERR_UNSUPPORTED;
    auto kern = filter_simt_kernel<TQ, ADJ>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return IFDK_ERR_CUDA;
    const int gx = (g.nu + kOutPerBlock - 1) / kOutPerBlock;
    for (long long r0 = 0; r0 < rows; r0 += chunk) {
        const long long nr = rows - r0 < chunk ? rows - r0 : chunk;
        kern<<<dim3(gx, (unsigned)((nr + kRows - 1) / kRows)), kFThreads, smem, stream>>>(
            E + r0 * g.nu, static_cast<TQ *>(Q) + r0 * g.nu, p->d_fcos, p->d_taps, g.nu, g.nv, nr);
        if (cudaGetLastError() != cudaSuccess) return IFDK_ERR_CUDA;
    }
    return IFDK_OK;
}

}  // namespace

int launch_filter(ifdk_plan_s *p, const float *E, void *Q, int q_dtype, int split_terms, bool adjoint,
                  cudaStream_t stream)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    (void)split_terms;
    if (adjoint) return launch_simt<float, true>(p, E, Q, stream);
    switch (q_dtype) {
    case IFDK_F32: return launch_simt<float, false>(p, E, Q, stream);
    case IFDK_F16: return launch_simt<__half, false>(p, E, Q, stream);
    default: return launch_simt<__nv_bfloat16, false>(p, E, Q, stream);
    }
}

}  // namespace ifdk
