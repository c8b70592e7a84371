// Output stage of Algorithm 4: I <- reshape(I~).  The back-projectors
// accumulate the k-major volume I~ [nx][ny][nz] (k fastest, Sec. 3.3, data
// layout); the paper's output is the i-major volume, stored as nz slices of
// nx x ny (Sec. 4, the volume written as slices).  This is a plain transpose
// per j, HBM-bound: every element is read once and written once.
//
// A block owns a 64 (i) x 64 (k) tile of one j: reads are 32 consecutive k of
// one i per warp instruction (128 B), writes 32 consecutive i of one k; the
// tile passes through shared memory with a padded row so that both phases are
// free of bank conflicts.  16-bit outputs round to nearest even.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ifdk_internal.h"

namespace ifdk {
namespace {

constexpr int kSlTile = 64;
constexpr int kSlThreads = 256;

template <typename T> __device__ __forceinline__ T from_f32(float x);
template <> __device__ __forceinline__ float from_f32<float>(float x) { return x; }
template <> __device__ __forceinline__ __half from_f32<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

struct SlArgs {
    const float *vol;
    void *out;
    int nx, ny, nz, k_begin, k_count;
};

template <typename T>
__global__ void __launch_bounds__(kSlThreads) slices_kernel(const SlArgs a)
{
    __shared__ float tile[kSlTile][kSlTile + 1];   // [i][k], padded
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i0 = blockIdx.x * kSlTile, kk0 = blockIdx.y * kSlTile, j = blockIdx.z;
    const int ni = min(kSlTile, a.nx - i0), nk = min(kSlTile, a.k_count - kk0);

    // read: warp w takes rows i = w, w + 8, ...; lanes run along k (two halves of 32)
#pragma unroll
    for (int r = 0; r < kSlTile / 8; ++r) {
        const int ii = warp + 8 * r;
        if (ii < ni) {
            const float *col = a.vol + ((size_t)(i0 + ii) * a.ny + j) * (size_t)a.nz + a.k_begin + kk0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kk = lane + 32 * h;
                if (kk < nk) tile[ii][kk] = __ldcs(col + kk);
            }
        }
    }
    __syncthreads();

    // write: warp w takes slices kk = w, w + 8, ...; lanes run along i
    T *out = static_cast<T *>(a.out);
#pragma unroll
    for (int r = 0; r < kSlTile / 8; ++r) {
        const int kk = warp + 8 * r;
        if (kk < nk) {
            T *row = out + ((size_t)(kk0 + kk) * a.ny + j) * (size_t)a.nx + i0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ii = lane + 32 * h;
                if (ii < ni) __stcs(row + ii, from_f32<T>(tile[ii][kk]));
            }
        }
    }
}

}  // namespace

int launch_volume_slices(ifdk_plan_s *p, const float *vol, void *out, int out_dtype, int k_begin, int k_count,
                         cudaStream_t stream)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    const ifdk_geometry &g = p->g;
    SlArgs a{vol, out, g.nx, g.ny, g.nz, k_begin, k_count};
    const dim3 grid((g.nx + kSlTile - 1) / kSlTile, (k_count + kSlTile - 1) / kSlTile, g.ny);
    if (grid.y > 65535 || grid.z > 65535) return IFDK_ERR_UNSUPPORTED;
    switch (out_dtype) {
    case IFDK_F32: slices_kernel<float><<<grid, kSlThreads, 0, stream>>>(a); break;
    case IFDK_F16: slices_kernel<__half><<<grid, kSlThreads, 0, stream>>>(a); break;
    case IFDK_BF16: slices_kernel<__nv_bfloat16><<<grid, kSlThreads, 0, stream>>>(a); break;
    default: return IFDK_ERR_INVALID;
    }
    return cudaGetLastError() == cudaSuccess ? IFDK_OK : IFDK_ERR_CUDA;
}

}  // namespace ifdk
