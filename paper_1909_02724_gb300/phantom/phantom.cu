// Input generator: exact line integrals of additive ellipsoids along the cone
// beam rays, in FP32 on the GPU (for workloads too large for the FP64 CPU
// generator in __init__.py, which it is checked against).  No reconstruction
// arithmetic lives here.  Built into its own shared library.
//
// Scanner (world frame): source S = (-d sin b, -d cos b, 0); the ray to pixel
// (iu, iv) has direction D n + a e_u + b e_v with n = (sin b, cos b, 0),
// e_u = (cos b, -sin b, 0), e_v = (0, 0, -1), a = (iu - uc) Du, b = (iv - vc) Dv.
// Per ellipsoid (centre c, M = diag(1/axes) R^T, density rho) the quadratic is
// solved about the point of the ray nearest the centre.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

namespace {

struct Ell {
    float m[9];
    float c[3];
    float rho;
    float pad[3];
};

struct ViewG {
    float sx, sy;      // source XY
    float cb, sb;      // cos, sin of the view angle
};

constexpr int kMaxEll = 1024;

__global__ void __launch_bounds__(256) phantom_kernel(const Ell *__restrict__ ell, int n_ell,
                                                      const ViewG *__restrict__ views, float sdd,
                                                      int nu, int nv, float du, float dv, float uc,
                                                      float vc, float *__restrict__ E)
{
    __shared__ Ell se[64];
    const int iu = blockIdx.x * 16 + (threadIdx.x & 15);
    const int iv = blockIdx.y * 16 + (threadIdx.x >> 4);
    const int s = blockIdx.z;
    const ViewG vg = views[s];
    const float a = ((float)iu - uc) * du, b = ((float)iv - vc) * dv;
    // direction = D n + a e_u + b e_v
    float dx = sdd * vg.sb + a * vg.cb;
    float dy = sdd * vg.cb - a * vg.sb;
    float dz = -b;
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv; dy *= inv; dz *= inv;
    float total = 0.0f;
    for (int e0 = 0; e0 < n_ell; e0 += 64) {
        __syncthreads();
        const int ne = min(64, n_ell - e0);
        for (int t = threadIdx.x; t < ne * 16; t += blockDim.x)
            reinterpret_cast<float *>(se)[t] = reinterpret_cast<const float *>(ell + e0)[t];
        __syncthreads();
        for (int e = 0; e < ne; ++e) {
            const Ell &q = se[e];
            // w = c - S; rel = (w . d) d - w  (the nearest point minus the centre)
            const float wx = q.c[0] - vg.sx, wy = q.c[1] - vg.sy, wz = q.c[2];
            const float t0 = wx * dx + wy * dy + wz * dz;
            const float rx = t0 * dx - wx, ry = t0 * dy - wy, rz = t0 * dz - wz;
            const float spx = q.m[0] * rx + q.m[1] * ry + q.m[2] * rz;
            const float spy = q.m[3] * rx + q.m[4] * ry + q.m[5] * rz;
            const float spz = q.m[6] * rx + q.m[7] * ry + q.m[8] * rz;
            const float dpx = q.m[0] * dx + q.m[1] * dy + q.m[2] * dz;
            const float dpy = q.m[3] * dx + q.m[4] * dy + q.m[5] * dz;
            const float dpz = q.m[6] * dx + q.m[7] * dy + q.m[8] * dz;
            const float A = dpx * dpx + dpy * dpy + dpz * dpz;
            const float B = spx * dpx + spy * dpy + spz * dpz;
            const float C = spx * spx + spy * spy + spz * spz - 1.0f;
            const float disc = B * B - A * C;
            if (disc > 0.0f) total += q.rho * 2.0f * sqrtf(disc) / A;
        }
    }
    if (iu < nu && iv < nv) E[((size_t)s * nv + iv) * nu + iu] = total;
}

}  // namespace

extern "C" {

// Line integrals of the packed ellipsoid set (n_ell rows of 16 doubles:
// centre(3), 1/axes(3), rotation row-major(9), rho) for views
// [view_begin, view_begin + view_count) into E (device FP32
// [view_count][nv][nu]).  Returns 0 on success, -1 on a bad argument, -4 on
// a CUDA error.  Synchronous with respect to the host.
int ifdk_phantom_project(const double *ell, int n_ell, double sid, double sdd, int nu, int nv, double du,
                         double dv, double off_u, double off_v, const double *angles, int view_begin,
                         int view_count, float *E, void *stream)
{
    if (!ell || !angles || !E || n_ell < 1 || n_ell > kMaxEll || nu < 1 || nv < 1 || view_count < 1 ||
        view_count > 65535)
        return -1;
    std::vector<Ell> he(n_ell);
    for (int e = 0; e < n_ell; ++e) {
        const double *r = ell + 16 * e;
        // M = diag(1/axes) R^T: row a of M is (1/axis_a) * column a of R
        for (int ra = 0; ra < 3; ++ra)
            for (int cc = 0; cc < 3; ++cc) he[e].m[3 * ra + cc] = (float)(r[3 + ra] * r[6 + 3 * cc + ra]);
        for (int q = 0; q < 3; ++q) he[e].c[q] = (float)r[q];
        he[e].rho = (float)r[15];
        he[e].pad[0] = he[e].pad[1] = he[e].pad[2] = 0.0f;
    }
    std::vector<ViewG> hv(view_count);
    for (int s = 0; s < view_count; ++s) {
        const double bb = angles[view_begin + s];
        hv[s].sx = (float)(-sid * std::sin(bb));
        hv[s].sy = (float)(-sid * std::cos(bb));
        hv[s].cb = (float)std::cos(bb);
        hv[s].sb = (float)std::sin(bb);
    }
    Ell *de = nullptr;
    ViewG *dvw = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMalloc(&de, sizeof(Ell) * n_ell) != cudaSuccess) return -4;
    if (cudaMalloc(&dvw, sizeof(ViewG) * view_count) != cudaSuccess) { cudaFree(de); return -4; }
    int rc = 0;
    if (cudaMemcpy(de, he.data(), sizeof(Ell) * n_ell, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dvw, hv.data(), sizeof(ViewG) * view_count, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = -4;
    if (rc == 0) {
        const float uc = (float)((nu - 1) / 2.0 + off_u / du), vc = (float)((nv - 1) / 2.0 + off_v / dv);
        dim3 grid((nu + 15) / 16, (nv + 15) / 16, view_count);
        phantom_kernel<<<grid, 256, 0, st>>>(de, n_ell, dvw, (float)sdd, nu, nv, (float)du, (float)dv, uc, vc, E);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) rc = -4;
    }
    cudaFree(de);
    cudaFree(dvw);
    return rc;
}

}  // extern "C"
