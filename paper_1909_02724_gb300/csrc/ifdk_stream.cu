// ifdk_backproject_host: back-projection of filtered views that live in host
// memory, streamed to the device in view chunks while the back-projection
// runs (Sec. 4 of the iFDK paper overlaps the host-to-device transfer with
// back-projection, so that T_H2D hides inside T_bp).
//
// Two staging halves on the device.  Chunk c goes to half c & 1:
//   copy stream:  wait ev_bp[h] (the back-projection of chunk c - 2 is done
//                 reading the half), one copy of the chunk's views (strided,
//                 cudaMemcpy2DAsync, when the plan's detector rows are a part
//                 of each host view), record ev_copy[h];
//   `stream`:     wait ev_copy[h], back-project the chunk from the half
//                 (ifdk_backproject_views addressing), record ev_bp[h].
// The first copy waits for an event recorded on `stream` at entry, so it
// never overwrites staging that earlier work on `stream` still reads.  Every
// copy is waited for by a later back-projection on `stream`, so work issued
// on `stream` after this call sees every copy complete.
#include "ifdk_device.cuh"
#include "ifdk_internal.h"

using namespace ifdk;

extern "C" int ifdk_backproject_host(ifdk_plan p, const void *Q_host, int q_dtype, int host_nv, int host_row0,
                                     int view_begin, int view_count, int chunk_views, void *staging,
                                     size_t staging_bytes, float *vol, void *stream)
{
    if (!p || !Q_host || !staging) return IFDK_ERR_INVALID;
    int rc = check_backproject_args(p, staging, q_dtype, view_begin, view_count, vol);
    if (rc != IFDK_OK) return rc;
    const ifdk_geometry &g = p->g;
    if (chunk_views < 1 || host_row0 < 0 || host_nv < g.nv || host_row0 > host_nv - g.nv) return IFDK_ERR_INVALID;
    if ((uintptr_t)staging & 255) return IFDK_ERR_ALIGNMENT;
    const size_t es = q_dtype == IFDK_F32 ? 4 : 2;
    const size_t view_bytes = (size_t)g.nv * g.nu * es;
    const size_t half_bytes = (size_t)chunk_views * view_bytes;
    if (staging_bytes < 2 * half_bytes) return IFDK_ERR_INVALID;
    if (view_count == 0) return IFDK_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;

    cudaStream_t s = (cudaStream_t)stream, cs = p->copy_stream;
    const size_t host_view_bytes = (size_t)host_nv * g.nu * es;
    const unsigned char *src0 = static_cast<const unsigned char *>(Q_host) + (size_t)host_row0 * g.nu * es;
    if (cudaEventRecord(p->ev_start, s) != cudaSuccess || cudaStreamWaitEvent(cs, p->ev_start, 0) != cudaSuccess)
        return IFDK_ERR_CUDA;
    const int nchunks = (view_count + chunk_views - 1) / chunk_views;
    for (int c = 0; c < nchunks; ++c) {
        const int h = c & 1;
        const int v0 = view_begin + c * chunk_views;
        const int nvc = std::min(chunk_views, view_begin + view_count - v0);
        unsigned char *dst = static_cast<unsigned char *>(staging) + h * half_bytes;
        if (c >= 2 && cudaStreamWaitEvent(cs, p->ev_bp[h], 0) != cudaSuccess) return IFDK_ERR_CUDA;
        const unsigned char *src = src0 + (size_t)v0 * host_view_bytes;
        const cudaError_t ce =
            host_nv == g.nv ? cudaMemcpyAsync(dst, src, (size_t)nvc * view_bytes, cudaMemcpyHostToDevice, cs)
                            : cudaMemcpy2DAsync(dst, view_bytes, src, host_view_bytes, view_bytes, (size_t)nvc,
                                                cudaMemcpyHostToDevice, cs);
        if (ce != cudaSuccess || cudaEventRecord(p->ev_copy[h], cs) != cudaSuccess || cudaStreamWaitEvent(s, p->ev_copy[h], 0) != cudaSuccess)
            return IFDK_ERR_CUDA;
        rc = launch_backproject(p, dst, q_dtype, v0, nvc, v0, nvc, vol, s);
        if (rc != IFDK_OK) return rc;
        if (cudaEventRecord(p->ev_bp[h], s) != cudaSuccess) return IFDK_ERR_CUDA;
    }
    return IFDK_OK;
}
