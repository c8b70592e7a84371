// ifdk_filter_noalloc: the tensor-core filtering stage for callers that
// cannot allocate device memory.  Its split-operand workspace is a fixed
// file-scope device array instead of a caller buffer; everything else is the
// ifdk_filter tensor-core path, unchanged.
//
// The array is part of the library's device image: every GPU on which the
// library's code is loaded holds it (kStaticWorkspaceBytes) until the process
// exits.  In host code `g_filter_workspace` is only a stand-in for the
// symbol, so its device address is looked up with cudaGetSymbolAddress, once
// per device, with that device current, and cached.
#include <mutex>

#include "ifdk_device.cuh"
#include "ifdk_internal.h"

namespace {

constexpr size_t kStaticWorkspaceBytes = (size_t)16 << 20;   // 16 MiB
__device__ __align__(256) unsigned char g_filter_workspace[kStaticWorkspaceBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_address[kMaxDevices];   // device address of g_filter_workspace, per device

// Device address of the array on the current device (looked up on first use).
int workspace_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) return IFDK_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_address[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_filter_workspace) != cudaSuccess || !p) {
            cudaGetLastError();
            return IFDK_ERR_CUDA;
        }
        g_address[dev] = p;
    }
    *out = g_address[dev];
    return IFDK_OK;
}

}  // namespace

extern "C" int ifdk_filter_noalloc(ifdk_plan p, const float *E, void *Q, int q_dtype, int split_terms,
                                   void *stream)
{
    using namespace ifdk;
    if (!p || !E || !Q) return IFDK_ERR_INVALID;
    if (q_dtype != IFDK_F32 && q_dtype != IFDK_F16 && q_dtype != IFDK_BF16) return IFDK_ERR_INVALID;
    if (split_terms < 1 || split_terms > 3) return IFDK_ERR_INVALID;
    // the fixed array must hold at least one 128-row tile of split operands
    if (filter_workspace_min(p, split_terms) > kStaticWorkspaceBytes) return IFDK_ERR_UNSUPPORTED;
    if (((uintptr_t)E & 15) || ((uintptr_t)Q & 15)) return IFDK_ERR_ALIGNMENT;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    void *ws = nullptr;
    const int rc = workspace_address(dev, &ws);
    if (rc != IFDK_OK) return rc;
    return launch_filter_tc(p, E, Q, q_dtype, split_terms, ws, kStaticWorkspaceBytes, (cudaStream_t)stream);
}
