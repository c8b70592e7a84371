// Filtering stage (Algorithm 1 of the iFDK paper): cosine weight F_cos then
// the Ram-Lak ramp convolution of every detector row, the exact linear (zero
// padded) convolution truncated to Nu outputs, as a dense Toeplitz product.
//
// FP32 SIMT kernel.  The forward filter sums by parts: with w = F_cos E (0
// outside the row), d(m) = w(m) - w(m-1) for m in [0, nu] and the running tap
// sum g(n) = sum_{j <= n} h(j), Q(n) = sum_m g(n - m) d(m), which avoids the
// ~1400x cancellation of the direct sum at 2048 pixels (d is formed from a
// double-float w).  The adjoint (gradient) is the direct transpose,
// F_cos . (T^T q) with T[n][m] = h(n - m).
//
// A block computes 1024 consecutive outputs of kRows rows; the input rows
// and the taps the block needs sit in shared memory; every thread keeps 4
// consecutive outputs x kRows rows in registers and slides a 4-tap window
// down the Toeplitz diagonal; the epilogue casts to the storage type.
#include "ifdk_device.cuh"
#include "ifdk_internal.h"

namespace ifdk {
namespace {

constexpr int kRows = 4;          // rows per block
constexpr int kOutPerThread = 4;  // consecutive outputs per thread
constexpr int kFThreads = 256;
constexpr int kOutPerBlock = kFThreads * kOutPerThread;

// Weighted sample w(m) = E F_cos as a double-float p + c; 0 outside [0, nu).
// srow (short scan, else nullptr): the view's per-column redundancy weights.
__device__ __forceinline__ void weighted_df(const float *__restrict__ Erow, const float *__restrict__ fh_row,
                                            const float *__restrict__ fl_row, const float *__restrict__ srow, int m,
                                            int nu, float &p, float &c)
{
    p = 0.0f;
    c = 0.0f;
    if (m >= 0 && m < nu) {
        const float x = __ldg(Erow + m), fh = __ldg(fh_row + m);
        p = x * fh;
        c = fmaf(x, __ldg(fl_row + m), fmaf(x, fh, -p));
        if (srow) df_scale(p, c, __ldg(srow + m));
    }
}

// Forward: len = nu + 1 inputs d(m), taps = g with tap(n) = taps[n + nu] for
// n in [-nu, nu - 1].  Adjoint: len = nu inputs q(m), taps = h with
// tap(n) = taps[n + nu - 1] for |n| < nu.
template <typename TQ, bool ADJ>
__global__ void __launch_bounds__(kFThreads)
    filter_simt_kernel(const float *__restrict__ E, TQ *__restrict__ Q, const float *__restrict__ fcos,
                       const float *__restrict__ fcos_lo, const float *__restrict__ taps, int nu, int nv,
                       long long rows, unsigned int *view_max, int view0, const float *__restrict__ sweight)
{
    extern __shared__ float sm[];
    const int len = ADJ ? nu : nu + 1;
    float *w = sm;                        // [kRows][len] input rows
    float *hs = sm + kRows * len;         // taps window, see below
    const int n_lo = blockIdx.x * kOutPerBlock;
    const long long r0 = (long long)blockIdx.y * kRows;

    for (int r = 0; r < kRows; ++r) {
        const long long row = r0 + r;
        for (int m = threadIdx.x; m < len; m += kFThreads) {
            float x = 0.0f;
            if (row < rows) {
                if (ADJ) {
                    x = __ldg(E + row * nu + m);
                } else {
                    const size_t vo = (size_t)(row % nv) * nu;
                    const float *srow = sweight ? sweight + (size_t)(view0 + row / nv) * nu : nullptr;
                    float p1, c1, p0, c0;
                    weighted_df(E + row * nu, fcos + vo, fcos_lo + vo, srow, m, nu, p1, c1);
                    weighted_df(E + row * nu, fcos + vo, fcos_lo + vo, srow, m - 1, nu, p0, c0);
                    const float s = p1 - p0, bb = s - p1;
                    const float err = (p1 - (s - bb)) + (-p0 - bb);   // s + err = p1 - p0 exactly
                    x = s + (err + (c1 - c0));
                }
            }
            w[r * len + m] = x;
        }
    }
    // hs[t] = tap(n) with n = t - 4 + n_lo - (len - 1), for n in the range the block uses.
    const int hlen = kOutPerBlock + len + 4;
    for (int t = threadIdx.x; t < hlen; t += kFThreads) {
        const int n = t - 4 + n_lo - (len - 1);
        hs[t] = ADJ ? ((n > -nu && n < nu) ? __ldg(taps + n + nu - 1) : 0.0f)
                    : ((n >= -nu && n < nu) ? __ldg(taps + n + nu) : 0.0f);
    }
    __syncthreads();

    const int n0 = n_lo + threadIdx.x * kOutPerThread;
    // past the row end: nothing to compute, unless the warp's per-view maximum
    // needs every lane (the loop below then only reads the tap window)
    if (n0 >= nu && view_max == nullptr) return;
    float acc[kRows][kOutPerThread];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int q = 0; q < kOutPerThread; ++q) acc[r][q] = 0.0f;
    // output n0+q at input m uses tap(n0 + q - m) = hs[base + q - m]
    const int base = threadIdx.x * kOutPerThread + len - 1 + 4;
    float h0 = hs[base], h1 = hs[base + 1], h2 = hs[base + 2], h3 = hs[base + 3];
    for (int m = 0; m < len; ++m) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const float x = w[r * len + m];
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
                if (ADJ) {
                    y *= __ldg(fcos + (row % nv) * nu + n);
                    if (sweight) y *= __ldg(sweight + (size_t)(view0 + row / nv) * nu + n);
                }
                Q[row * nu + n] = Storage<TQ>::from_float(y);
            }
        }
    }
    if (!ADJ && view_max != nullptr) {
        // every lane of the warp holds the same kRows rows: per row, the lanes'
        // maxima (FP32, before the cast) meet by a butterfly of warp shuffles
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const long long row = r0 + r;
            uint32_t m = 0u;
#pragma unroll
            for (int q = 0; q < kOutPerThread; ++q)
                if (n0 + q < nu && row < rows) m = max(m, __float_as_uint(acc[r][q]) & 0x7fffffffu);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, d));
            if ((threadIdx.x & 31) == 0 && row < rows && m != 0u) atomicMax(view_max + view0 + (int)(row / nv), m);
        }
    }
}

// E, Q: views [view_begin, view_begin + view_count) (row 0 = row 0 of view view_begin)
template <typename TQ, bool ADJ>
int launch_simt(ifdk_plan_s *p, const float *E, void *Q, cudaStream_t stream, unsigned int *view_max, int view_begin,
                int view_count)
{
    const ifdk_geometry &g = p->g;
    const long long rows = (long long)view_count * g.nv;
    const int len = ADJ ? g.nu : g.nu + 1;
    const size_t smem = sizeof(float) * ((size_t)kRows * len + kOutPerBlock + len + 4);
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
            E + r0 * g.nu, static_cast<TQ *>(Q) + r0 * g.nu, p->d_fcos, p->d_fcos_lo, ADJ ? p->d_taps : p->d_gsum,
            g.nu, g.nv, nr, view_max, view_begin + (int)(r0 / g.nv), p->d_sweight);
        if (cudaGetLastError() != cudaSuccess) return IFDK_ERR_CUDA;
    }
    return IFDK_OK;
}

}  // namespace

int launch_filter(ifdk_plan_s *p, const float *E, void *Q, int q_dtype, int split_terms, bool adjoint,
                  cudaStream_t stream, unsigned int *view_max, int view_begin, int view_count)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    (void)split_terms;
    if (view_count < 0) view_count = p->g.np - view_begin;
    if (view_count == 0) return IFDK_OK;
    const int b = view_begin, n = view_count;
    if (adjoint) return launch_simt<float, true>(p, E, Q, stream, nullptr, b, n);
    switch (q_dtype) {
    case IFDK_F32: return launch_simt<float, false>(p, E, Q, stream, view_max, b, n);
    case IFDK_F16: return launch_simt<__half, false>(p, E, Q, stream, view_max, b, n);
    default: return launch_simt<__nv_bfloat16, false>(p, E, Q, stream, view_max, b, n);
    }
}

}  // namespace ifdk
