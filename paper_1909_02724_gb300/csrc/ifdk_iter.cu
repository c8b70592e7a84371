// Element-wise steps of the iterative solvers that reuse the back-projector and
// its adjoint (the paper names SART and MLEM as such users, Sec. 1 and Sec. 6):
//
//   SART (Andersen & Kak 1984), over a subset S of the views:
//     r = (p - A x) / R          on the rays of S (R = A 1; 0 where R = 0)
//     x <- x + lam (A_S^T r) / C_S                (C_S = A_S^T 1; x kept where C_S = 0)
//   MLEM (Shepp & Vardi 1982; ordered subsets, Hudson & Larkin 1994):
//     r = p / (A x)              on the rays of S (0 where A x = 0)
//     x <- x (A_S^T r) / C_S                      (x kept where C_S = 0)
//
// A is ifdk_project and A^T the back-projection; the two kernels here are the
// ray-space ratio (which also clears the forward projection it read, so that
// the next subset's projection accumulates into zeros) and the volume update
// (which clears the back-projection it read, likewise).  Both are one
// streaming pass over HBM: float4 accesses when every pointer is 16-byte
// aligned, scalar ones otherwise; the divisions are IEEE (no fast math).
#include "ifdk_device.cuh"
#include "ifdk_internal.h"

namespace ifdk {
namespace {

__device__ __forceinline__ float ratio_of(int method, float p, float ax, float r)
{
    if (method == IFDK_SART) return r > 0.0f ? (p - ax) / r : 0.0f;
    return ax > 0.0f ? p / ax : 0.0f;
}

__device__ __forceinline__ float update_of(int method, float x, float u, float c, float lam, int nonneg)
{
    if (!(c > 0.0f)) return x;
    float y;
    if (method == IFDK_SART) {
        y = fmaf(lam, u / c, x);
        if (nonneg) y = fmaxf(y, 0.0f);
    } else {
        y = x * u / c;
    }
    return y;
}

__global__ void __launch_bounds__(256) ratio_kernel(int method, const float *__restrict__ Pm, float *Ax,
                                                   const float *__restrict__ R, float *__restrict__ out, size_t n,
                                                   bool vec)
{
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
    size_t done = 0;
    if (vec) {
        const size_t n4 = n / 4;
        for (size_t i = t0; i < n4; i += step) {
            const float4 p = __ldcs(reinterpret_cast<const float4 *>(Pm) + i);
            const float4 a = reinterpret_cast<const float4 *>(Ax)[i];
            const float4 r = R ? __ldcs(reinterpret_cast<const float4 *>(R) + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 o;
            o.x = ratio_of(method, p.x, a.x, r.x);
            o.y = ratio_of(method, p.y, a.y, r.y);
            o.z = ratio_of(method, p.z, a.z, r.z);
            o.w = ratio_of(method, p.w, a.w, r.w);
            reinterpret_cast<float4 *>(out)[i] = o;
            reinterpret_cast<float4 *>(Ax)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        done = 4 * n4;
    }
    for (size_t i = done + t0; i < n; i += step) {
        out[i] = ratio_of(method, Pm[i], Ax[i], R ? R[i] : 0.0f);
        Ax[i] = 0.0f;
    }
}

__global__ void __launch_bounds__(256) update_kernel(int method, float *x, float *U, const float *__restrict__ C,
                                                    size_t n, float lam, int nonneg, bool vec)
{
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
    size_t done = 0;
    if (vec) {
        const size_t n4 = n / 4;
        for (size_t i = t0; i < n4; i += step) {
            float4 v = reinterpret_cast<float4 *>(x)[i];
            const float4 u = reinterpret_cast<const float4 *>(U)[i];
            const float4 c = __ldcs(reinterpret_cast<const float4 *>(C) + i);
            v.x = update_of(method, v.x, u.x, c.x, lam, nonneg);
            v.y = update_of(method, v.y, u.y, c.y, lam, nonneg);
            v.z = update_of(method, v.z, u.z, c.z, lam, nonneg);
            v.w = update_of(method, v.w, u.w, c.w, lam, nonneg);
            reinterpret_cast<float4 *>(x)[i] = v;
            reinterpret_cast<float4 *>(U)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        done = 4 * n4;
    }
    for (size_t i = done + t0; i < n; i += step) {
        x[i] = update_of(method, x[i], U[i], C[i], lam, nonneg);
        U[i] = 0.0f;
    }
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

unsigned grid_for(const ifdk_plan_s *p, size_t n)
{
    const size_t want = (n / 4 + 255) / 256 + 1, cap = (size_t)(p->n_sm > 0 ? p->n_sm : 152) * 16;
    return (unsigned)(want < cap ? want : cap);
}

}  // namespace
}  // namespace ifdk

using namespace ifdk;

extern "C" int ifdk_iter_ratio(ifdk_plan p, int method, const float *Pm, float *Ax, const float *R, float *out,
                               int view_count, void *stream)
{
    if (!p || (method != IFDK_SART && method != IFDK_MLEM)) return IFDK_ERR_INVALID;
    if (view_count < 0 || view_count > p->g.np) return IFDK_ERR_INVALID;
    if (view_count == 0) return IFDK_OK;
    if (!Pm || !Ax || !out || (method == IFDK_SART && !R)) return IFDK_ERR_INVALID;
    if (((uintptr_t)Pm | (uintptr_t)Ax | (uintptr_t)R | (uintptr_t)out) & 3) return IFDK_ERR_ALIGNMENT;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    const size_t n = (size_t)view_count * p->g.nv * p->g.nu;
    const bool vec = aligned16(Pm) && aligned16(Ax) && aligned16(out) && (!R || aligned16(R));
    ratio_kernel<<<grid_for(p, n), 256, 0, (cudaStream_t)stream>>>(method, Pm, Ax, method == IFDK_SART ? R : nullptr,
                                                                  out, n, vec);
    return cudaGetLastError() == cudaSuccess ? IFDK_OK : IFDK_ERR_CUDA;
}

extern "C" int ifdk_iter_update(ifdk_plan p, int method, float *x, float *U, const float *C, float lambda,
                                int nonneg, void *stream)
{
    if (!p || (method != IFDK_SART && method != IFDK_MLEM) || !x || !U || !C) return IFDK_ERR_INVALID;
    if (nonneg != 0 && nonneg != 1) return IFDK_ERR_INVALID;
    if (((uintptr_t)x | (uintptr_t)U | (uintptr_t)C) & 3) return IFDK_ERR_ALIGNMENT;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    const size_t n = (size_t)p->g.nx * p->g.ny * p->g.nz;
    const bool vec = aligned16(x) && aligned16(U) && aligned16(C);
    update_kernel<<<grid_for(p, n), 256, 0, (cudaStream_t)stream>>>(method, x, U, C, n, lambda, nonneg, vec);
    return cudaGetLastError() == cudaSuccess ? IFDK_OK : IFDK_ERR_CUDA;
}
