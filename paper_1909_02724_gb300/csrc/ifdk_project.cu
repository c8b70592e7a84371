// Adjoint of the back-projection: the transpose of Algorithm 4 / Algorithm 3.
// Every voxel value is splatted with weight w_s f^2 times its bilinear
// coefficients onto the four taps of every view (FP32 atomics; a thread sums
// the taps its z-run puts on the same detector row before the atomic).  The per
// (column, view) terms are formed once and reused over the thread's z-run,
// exactly as in the back-projection.
#include "ifdk_device.cuh"
#include "ifdk_internal.h"

namespace ifdk {
namespace {

constexpr int kProjZ = 16;

struct ProjArgs {
    const float *vol;
    float *P;
    const ViewTerms *terms;
    int nx, ny, nz, nu, nv, tiles_x;
    int view_begin, view_count;
    float cx, cy, cz, uc, vc;
};

__device__ __forceinline__ void splat(float *Ps, int nu, int nv, int iu, int iv, float val)
{
    if ((unsigned)iu < (unsigned)nu && (unsigned)iv < (unsigned)nv && val != 0.0f)
        atomicAdd(Ps + (size_t)iv * nu + iu, val);
}

// The view terms of the launch are staged in shared memory, kProjViews views at
// a time (one load per block instead of one dependent global load per thread
// and view).
constexpr int kProjViews = 512;

__global__ void __launch_bounds__(kThreads, 4) project_kernel(const ProjArgs a)
{
    __shared__ float4 sterms[kProjViews * 3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = (warp & 1) * 8 + (lane & 7), ty = (warp >> 1) * 4 + (lane >> 3);
    const int i = (blockIdx.x % a.tiles_x) * kTileX + tx, j = (blockIdx.x / a.tiles_x) * kTileY + ty;
    const bool inside = i < a.nx && j < a.ny;
    const int kb = blockIdx.y * kProjZ;
    float x[kProjZ];
    bool any = false;
#pragma unroll
    for (int z = 0; z < kProjZ; ++z) x[z] = 0.0f;
    if (inside) {
        const float *col = a.vol + ((size_t)i * a.ny + j) * (size_t)a.nz;
#pragma unroll
        for (int z = 0; z < kProjZ; ++z) {
            x[z] = kb + z < a.nz ? __ldg(col + kb + z) : 0.0f;
            any |= x[z] != 0.0f;
        }
    }
    // every thread of the block takes part in the staging (no early return before it)
    if (!__syncthreads_or(any)) return;
    const float ip = (float)i - a.cx, jp = (float)j - a.cy;
    for (int c0 = 0; c0 < a.view_count; c0 += kProjViews) {
        const int cn = min(kProjViews, a.view_count - c0);
        __syncthreads();
        const float4 *src = reinterpret_cast<const float4 *>(a.terms + a.view_begin + c0);
        for (int q = tid; q < 3 * cn; q += kThreads) sterms[q] = __ldg(src + q);
        __syncthreads();
        if (!any) continue;
        for (int c = 0; c < cn; ++c) {
            const int s = a.view_begin + c0 + c;
            const float4 t0 = sterms[3 * c], t1 = sterms[3 * c + 1], t2 = sterms[3 * c + 2];
            const float zc = fmaf(t1.y, ip, fmaf(t1.z, jp, t1.w));
            const float f = __frcp_rn(zc);
            const float u = fmaf(fmaf(t0.x, ip, fmaf(t0.y, jp, t0.z)), f, a.uc);
            if (!(u > -2.0f && u < a.nu + 1.0f)) continue;
            const float fu = floorf(u);
            const int iu = (int)fu;
            const float du = u - fu;
            const float W = t2.x * f * f;
            const float sig = t0.w * f;
            const float vb = fmaf(t1.x, f, a.vc);
            float *Ps = a.P + (size_t)s * a.nv * a.nu;
            // v is monotonic along the z-run, so consecutive voxels share detector rows
            // (one row per voxel at about one row per step): the taps of the two rows
            // last touched, pr and pr + 1, stay in registers and a row goes out (two
            // atomics) once no later voxel of the run can reach it
            bool pending = false;
            int pr = 0;
            float q00 = 0.0f, q01 = 0.0f, q10 = 0.0f, q11 = 0.0f;   // row pr: q00, q01; row pr + 1: q10, q11
    #pragma unroll
            for (int z = 0; z < kProjZ; ++z) {
                const float v = fmaf((float)(kb + z) - a.cz, sig, vb);
                if (!(v > -2.0f && v < a.nv + 1.0f)) continue;
                const float fv = floorf(v);
                const int iv = (int)fv;
                const float dv = v - fv;
                const float wv = W * x[z];
                const float lo = wv * (1.0f - dv), hi = wv * dv;
                const float a0 = lo * (1.0f - du), a1 = lo * du, b0 = hi * (1.0f - du), b1 = hi * du;
                if (pending && iv == pr) {
                    q00 += a0; q01 += a1; q10 += b0; q11 += b1;
                } else if (pending && iv == pr + 1) {
                    splat(Ps, a.nu, a.nv, iu, pr, q00);
                    splat(Ps, a.nu, a.nv, iu + 1, pr, q01);
                    q00 = q10 + a0; q01 = q11 + a1; q10 = b0; q11 = b1;
                    pr = iv;
                } else if (pending && iv == pr - 1) {
                    splat(Ps, a.nu, a.nv, iu, pr + 1, q10);
                    splat(Ps, a.nu, a.nv, iu + 1, pr + 1, q11);
                    q10 = q00 + b0; q11 = q01 + b1; q00 = a0; q01 = a1;
                    pr = iv;
                } else {
                    if (pending) {
                        splat(Ps, a.nu, a.nv, iu, pr, q00);
                        splat(Ps, a.nu, a.nv, iu + 1, pr, q01);
                        splat(Ps, a.nu, a.nv, iu, pr + 1, q10);
                        splat(Ps, a.nu, a.nv, iu + 1, pr + 1, q11);
                    }
                    q00 = a0; q01 = a1; q10 = b0; q11 = b1;
                    pr = iv;
                    pending = true;
                }
            }
            if (pending) {
                splat(Ps, a.nu, a.nv, iu, pr, q00);
                splat(Ps, a.nu, a.nv, iu + 1, pr, q01);
                splat(Ps, a.nu, a.nv, iu, pr + 1, q10);
                splat(Ps, a.nu, a.nv, iu + 1, pr + 1, q11);
            }
        }
    }
}

}  // namespace

int launch_project(ifdk_plan_s *p, const float *vol, float *P, int view_begin, int view_count,
                   cudaStream_t stream)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    const ifdk_geometry &g = p->g;
    ProjArgs a;
    a.vol = vol; a.P = P; a.terms = p->d_terms;
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.nu = g.nu; a.nv = g.nv;
    a.tiles_x = (g.nx + kTileX - 1) / kTileX;
    a.view_begin = view_begin; a.view_count = view_count;
    a.cx = (float)((g.nx - 1) / 2.0); a.cy = (float)((g.ny - 1) / 2.0); a.cz = (float)((g.nz - 1) / 2.0);
    a.uc = (float)p->uc; a.vc = (float)p->vc;
    const int tiles_y = (g.ny + kTileY - 1) / kTileY;
    const int zb = (g.nz + kProjZ - 1) / kProjZ;
    if (zb > 65535) return IFDK_ERR_UNSUPPORTED;
    project_kernel<<<dim3(a.tiles_x * tiles_y, zb), kThreads, 0, stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? IFDK_OK : IFDK_ERR_CUDA;
}

}  // namespace ifdk
