// Internal declarations of the ifdk library (not part of the C-ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ifdk.h"

namespace ifdk {

// Per-view FP32 projection terms.  P_s (Eq. 2) is formed in FP64 on the host
// and re-centred on the volume centre (i' = i - (nx-1)/2, ...) and on the
// principal point, so that for voxel (i', j', k'):
//   z = C0 i' + C1 j' + C3            (Theorem 3: no k' term)
//   u = uc + (A0 i' + A1 j' + A3) / z (Theorem 2: no k' term)
//   v = vc + (B2 k' + B3) / z         (no i', j' term in this geometry)
// w is the FDK constant dbeta_s d D / (2 du) of the view.
struct ViewTerms {
    float A0, A1, A3, B2;
    float B3, C0, C1, C3;
    float w, pad0, pad1, pad2;
};

// Fold (mirror-pair) back-projection: block tile and staging constants.
constexpr int kTileX = 16, kTileY = 16, kThreads = kTileX * kTileY;
constexpr int kPairs = 16;       // z pairs per thread (the thread's z-run)
constexpr int kViews = 4;        // max views per shared-memory chunk
constexpr int kFoldPitchS = 36;  // fold row pitch (elements; 4 mod 8 spreads banks) for widths <= 35
constexpr int kFoldPitchL = 52;  // ... and for widths <= 51
constexpr int kMargin = 1;       // window margin (pixels) on every side
constexpr int kGenZ = 16;        // z voxels per thread in the general kernel

struct BpLaunch {
    int path;          // 1 = fold (mirror pairs, TMA), 0 = general
    int fold_w;        // fold width (elements)
    int box_w, box_h;  // TMA box (elements, rows)
    int align;         // u alignment of the TMA box start (elements)
    int pitch;         // fold row pitch (elements)
    int views;         // views per shared-memory chunk
    size_t smem;       // dynamic shared memory bytes
    int grid_x, grid_y;
};

// Back-projection from packed (pre-folded) views: block tile as above, a ring
// of TMA stages of one view group each.
constexpr int kPkMaxStages = 8;
constexpr int kPkBoxS = 32, kPkBoxL = 48;   // box widths (elements) the kernel is built for
// z pairs per thread: 16 for single views; with half-turn view pairs (two
// columns' runs in registers) 16 for FP16 / BF16 storage and 12 for FP32,
// whose wider taps need the registers; with quarter-turn view quads (four
// columns' runs) 8.  A multiple of 4 (vector writes).
constexpr int pk_pairs(int nv, int q_dtype) { return nv == 4 ? 8 : (nv == 2 && q_dtype == IFDK_F32 ? 12 : 16); }
// resident blocks per SM the packed kernel is built for (registers) and sized for (shared memory)
constexpr int pk_blocks(int nv) { return nv >= 2 ? 2 : 3; }
// z pairs of the blocks after the full L-pair z-blocks (the volume's remainder)
constexpr int kPkTailL = 4;
// z-blocks of a packed launch: npairs / L full blocks, then tail blocks of kPkTailL pairs
constexpr int pk_zblocks(int npairs, int L) { return npairs / L + (npairs % L + kPkTailL - 1) / kPkTailL; }
// view split of the packed back-projection (small volumes): at most 16 partial
// volumes of at most 64 MiB together, each part at least 2 pairs (or views)
constexpr int kPkMaxSplits = 16, kPkSplitMinUnits = 2;
constexpr size_t kPkSplitBytes = (size_t)64 << 20;

struct PkLaunch {
    int path;          // 1 = packed mirror-pair kernel applies, 0 = not
    int nv;            // views per group: 1, or 2 (half-turn view pairs)
    int fold_w;        // window width (pixels)
    int bw, box_h;     // TMA box: elements (u), rows
    int align;         // u alignment of the box start (pixels)
    int stages;        // TMA stages in the ring
    int pairs;         // z pairs per thread
    size_t stage_bytes, smem;
    int grid_x, grid_y;
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled();  // cuTensorMapEncodeTiled through the runtime's driver entry point

inline size_t dtype_size(int t) { return t == IFDK_F32 ? 4 : 2; }

}  // namespace ifdk

struct ifdk_plan_s {
    ifdk_geometry g;                  // copy; angles/view_weights point into the vectors below
    std::vector<double> angles, weights;
    std::vector<ifdk::ViewTerms> terms;  // host copy of the FP32 table
    int device = 0;
    ifdk::ViewTerms *d_terms = nullptr;  // [np]
    float *d_fcos = nullptr;             // [nv][nu]
    float *d_fcos_lo = nullptr;          // [nv][nu], F_cos - (float)F_cos
    float *d_taps = nullptr;             // [2 nu - 1], index m + nu - 1
    float *d_gsum = nullptr;             // [2 nu], running tap sum g(m), index m + nu
    unsigned int *d_status = nullptr;    // device status word
    double uc = 0, vc = 0;               // principal point (pixels)
    int two_vc = 0;                      // 2 vc when it is an integer
    bool fold_ok = false;                // mirror-pair fold path applicable
    ifdk::BpLaunch bp[3];                // per storage type
    // packed views: rows r in [pk_row0, pk_row0 + pk_rows) pair row r with row 2 vc - r; a row
    // holds pk_nu elements (columns -1 .. nu - 1, rounded up to even) of 4 values each
    int pk_rows = 0, pk_nu = 0, pk_row0 = 0;   // pk_row0: detector row of packed row 0 (<= 0)
    float pk_wscale = 1.0f;              // power of two putting the largest FP16 weight in [1, 2)
    ifdk::PkLaunch pk[3], pk2[3], pk4[3];   // per storage type: single views / half-turn pairs / quarter-turn quads
    bool half_turn = false;              // view s + np/2 is view s turned by pi (exactly)
    bool quarter_turn = false;           // also view s + np/4 is view s turned by pi/2 (exactly)
    bool use_half_turn = true;           // caller switch (ifdk_set_view_pairing)
    bool use_quarter_turn = false;       // caller switch (ifdk_set_view_pairing mode 2)
    // short scan: 2 w(beta_s, gamma_u) per (view, column), [np][nu] (nullptr: full scan)
    float *d_sweight = nullptr;
    // view split: partial volumes [split_cap][split_stride] (allocated only for
    // small volumes), the caller's cap (0: automatic, 1: off) and the SM count
    float *d_split = nullptr;
    size_t split_stride = 0;
    int split_cap = 0, view_split_max = 0, n_sm = 0;
    unsigned long long wait_ns = 2000000000ull;
    int test_abort_group = -1;           // ifdk_set_test_abort (-1: off)
    // tensor-core filter: Toeplitz matrix as 3 BF16 planes [3][tc_npad][tc_kpad]
    int tc_kpad = 0, tc_npad = 0;
    uint16_t *d_tsplit = nullptr;
    // host streaming (ifdk_backproject_host): copy stream and, per staging
    // half, "copy landed" and "back-projection done" events
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copy[2] = {nullptr, nullptr}, ev_bp[2] = {nullptr, nullptr}, ev_start = nullptr;
};

// Implemented in ifdk_bp.cu / ifdk_filter.cu / ifdk_project.cu.
namespace ifdk {
void plan_backproject(ifdk_plan_s *p);
// Q holds views [q_view0, q_view0 + q_views) of [nv][nu] each.
int launch_backproject(ifdk_plan_s *p, const void *Q, int q_dtype, int view_begin, int view_count, int q_view0,
                       int q_views, float *vol, cudaStream_t stream);
// E, Q hold views [view_begin, view_begin + view_count) (view_count < 0: to the last view)
int launch_filter(ifdk_plan_s *p, const float *E, void *Q, int q_dtype, int split_terms, bool adjoint,
                  cudaStream_t stream, unsigned int *view_max = nullptr, int view_begin = 0, int view_count = -1);
int plan_filter_tc(ifdk_plan_s *p);
size_t filter_workspace_min(const ifdk_plan_s *p, int terms);
// view_max (optional): device [np] bits of max |Q| per view, zeroed by the caller
int launch_filter_tc(ifdk_plan_s *p, const float *E, void *Q, int q_dtype, int terms, void *ws, size_t ws_bytes,
                     cudaStream_t stream, unsigned int *view_max = nullptr, int view_begin = 0,
                     int view_count = -1);
int launch_project(ifdk_plan_s *p, const float *vol, float *P, int view_begin, int view_count,
                   cudaStream_t stream);
int launch_wait_selftest(ifdk_plan_s *p, unsigned long long ns, cudaStream_t stream);
int launch_volume_slices(ifdk_plan_s *p, const float *vol, void *out, int out_dtype, int k_begin, int k_count,
                         cudaStream_t stream);
// Packed views (ifdk_bp_packed.cu).
void plan_packed(ifdk_plan_s *p);
size_t packed_view_bytes(const ifdk_plan_s *p, int q_dtype);
// Q: [n_views][nv][nu] -> Qp: [n_views][pk_rows][pk_nu][4].
int launch_pack(ifdk_plan_s *p, const void *Q, int q_dtype, int n_views, void *Qp, cudaStream_t stream);
// Mirror pairs [pair0, pair0 + pcount) of the volume, written to a column of
// nz_out voxels (direct slab, then its mirror); pcount < 0: the whole volume.
struct PkZRange {
    int pair0 = 0, pcount = -1, nz_out = 0;
};
// Views [view_begin, view_begin + view_count) from packed views Qp that hold
// views [q_view0, q_view0 + q_views): half-turn pairs inside the range (if
// the plan pairs views) are back-projected together, the rest singly.
int launch_backproject_packed(ifdk_plan_s *p, const void *Qp, int q_dtype, int view_begin, int view_count,
                              int q_view0, int q_views, float *vol, cudaStream_t stream,
                              const PkZRange &zr = PkZRange{});
// Half-turn pairs (s, s + np/2) for s in [s_begin, s_begin + s_count); view s
// is packed view s - q_view0 and its partner packed view s - q_view0 + q_pair_off.
int launch_packed_pairs(ifdk_plan_s *p, const void *Qp, int q_dtype, int s_begin, int s_count, int q_view0,
                        int q_pair_off, int q_views, float *vol, cudaStream_t stream);
// Quarter-turn quads (s, s + np/4, s + np/2, s + 3np/4) for s in [s_begin, s_begin + s_count);
// view s + k np/4 is packed view s - q_view0 + k q_slot_off.
int launch_packed_quads(ifdk_plan_s *p, const void *Qp, int q_dtype, int s_begin, int s_count, int q_view0,
                        int q_slot_off, int q_views, float *vol, cudaStream_t stream);
// The views of [b, e) that pair up: s in [b, *m) with partners in [b + np/2, *m + np/2);
// the rest are [*m, b + np/2) and [*m + np/2, e).  *m = b when nothing pairs.
void split_half_turn(int np, int b, int e, int *m);
// View split of the packed back-projection: allocates the partial volumes at
// plan creation (small volumes only); the parts a launch over `units` pairs
// (pairs) or views uses.
int plan_view_split(ifdk_plan_s *p);
int packed_view_split(const ifdk_plan_s *p, int q_dtype, int units, int nv);
int check_backproject_args(const ifdk_plan_s *p, const void *Q, int q_dtype, int view_begin, int view_count,
                           const float *vol);
}  // namespace ifdk
