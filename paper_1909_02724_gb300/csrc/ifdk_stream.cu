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
// Packed path (staging large enough, packed views available): after the copy
// lands, the chunk is packed on `stream` into the half's packed part and the
// packed kernels run on it; with half-turn pairing the views that pair up go
// first, in pair chunks (views [s0, s0 + n) and [s0 + np/2, s0 + np/2 + n)
// copied side by side), then the unpaired views.
// The first copy waits for an event recorded on `stream` at entry, so it
// never overwrites staging that earlier work on `stream` still reads.  Every
// copy is waited for by a later back-projection on `stream`, so work issued
// on `stream` after this call sees every copy complete.
#include <vector>

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
    // packed path: the second part of the staging holds the packed halves
    const size_t pk_view = p->pk[q_dtype].path ? packed_view_bytes(p, q_dtype) : 0;
    const size_t pk_half = (size_t)chunk_views * pk_view;
    const bool packed = pk_view > 0 && staging_bytes >= 2 * (half_bytes + pk_half);
    struct Chunk { int s0, n, paired; };
    std::vector<Chunk> chunks;
    const int b = view_begin, e = view_begin + view_count, h = g.np / 2;
    int m = b;
    if (packed && p->use_half_turn && p->pk2[q_dtype].path && chunk_views >= 2) split_half_turn(g.np, b, e, &m);
    for (int s0 = b; s0 < m; s0 += chunk_views / 2) chunks.push_back({s0, std::min(chunk_views / 2, m - s0), 1});
    const int r0[2] = {m, m == b ? e : m + h}, r1[2] = {m == b ? e : b + h, e};
    for (int r = 0; r < 2; ++r)
        for (int s0 = r0[r]; s0 < r1[r]; s0 += chunk_views) chunks.push_back({s0, std::min(chunk_views, r1[r] - s0), 0});
    auto copy = [&](unsigned char *dst, int v0, int nvc) {
        const unsigned char *src = src0 + (size_t)v0 * host_view_bytes;
        return host_nv == g.nv ? cudaMemcpyAsync(dst, src, (size_t)nvc * view_bytes, cudaMemcpyHostToDevice, cs)
                               : cudaMemcpy2DAsync(dst, view_bytes, src, host_view_bytes, view_bytes, (size_t)nvc,
                                                   cudaMemcpyHostToDevice, cs);
    };
    for (size_t c = 0; c < chunks.size(); ++c) {
        const int hb = (int)(c & 1);
        const Chunk k = chunks[c];
        const int nq = k.paired ? 2 * k.n : k.n;   // views in the half
        unsigned char *dst = static_cast<unsigned char *>(staging) + hb * half_bytes;
        if (c >= 2 && cudaStreamWaitEvent(cs, p->ev_bp[hb], 0) != cudaSuccess) return IFDK_ERR_CUDA;
        cudaError_t ce = copy(dst, k.s0, k.n);
        if (ce == cudaSuccess && k.paired) ce = copy(dst + (size_t)k.n * view_bytes, k.s0 + h, k.n);
        if (ce != cudaSuccess || cudaEventRecord(p->ev_copy[hb], cs) != cudaSuccess ||
            cudaStreamWaitEvent(s, p->ev_copy[hb], 0) != cudaSuccess)
            return IFDK_ERR_CUDA;
        if (packed) {
            unsigned char *pk = static_cast<unsigned char *>(staging) + 2 * half_bytes + hb * pk_half;
            rc = launch_pack(p, dst, q_dtype, nq, pk, s);
            if (rc == IFDK_OK)
                rc = k.paired ? launch_packed_pairs(p, pk, q_dtype, k.s0, k.n, k.s0, k.n, nq, vol, s)
                              : launch_backproject_packed(p, pk, q_dtype, k.s0, k.n, k.s0, nq, vol, s);
        } else {
            rc = launch_backproject(p, dst, q_dtype, k.s0, k.n, k.s0, k.n, vol, s);
        }
        if (rc != IFDK_OK) return rc;
        if (cudaEventRecord(p->ev_bp[hb], s) != cudaSuccess) return IFDK_ERR_CUDA;
    }
    return IFDK_OK;
}
