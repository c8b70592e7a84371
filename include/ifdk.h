/*
 * ifdk.h -- C-ABI of the GB300-native FDK hot path of iFDK
 * (Chen, Wahib, Takizawa, Takano, Matsuoka, SC'19, arXiv 1909.02724).
 *
 * The library reconstructs a volume from circular cone-beam projections with
 * the FDK method: a filtering stage (cosine weight, then a Ram-Lak ramp
 * convolution along each detector row; Algorithm 1) and a voxel-driven
 * back-projection using the reduced-cost coordinate scheme of Algorithm 4
 * (Theorems 1-3).  It also provides the exact adjoint of the back-projection.
 *
 * Conventions shared by every call
 *   - Problem Nu x Nv x Np -> Nx x Ny x Nz (Sec. 2.3, definition I).
 *   - Projections E, Q, P: row-major [np][nv][nu] (U fastest), device memory.
 *   - Volume: row-major [nx][ny][nz] (k fastest: the k-major layout of
 *     Algorithm 4), device memory, FP32.
 *   - Voxel (i,j,k) sits at world X = dx (i-(nx-1)/2), Y = -dy (j-(ny-1)/2),
 *     Z = -dz (k-(nz-1)/2) + vol_off_z (the index flips of M0 in Eq. 2).
 *   - View s rotates the object by +angles[s] about Z (Mrot); the source sits
 *     at (-d sin b, -d cos b, 0); pixel (iu, iv) is centred at index position,
 *     principal point ((nu-1)/2 + off_u/du, (nv-1)/2 + off_v/dv) (M1).
 *   - Ownership: the caller owns every data buffer and stream.  A plan owns
 *     its geometry tables (view terms, F_cos, taps, the filter's split tap
 *     planes, the short-scan weights when set), a device status word, the
 *     partial volumes of the view split (small volumes only) and, for
 *     ifdk_backproject_host, a copy stream and events.
 *   - Asynchrony: filter / backproject / project enqueue kernels on `stream`
 *     (a cudaStream_t; NULL = the legacy default stream), allocate nothing,
 *     and do not synchronise.  Outputs of backproject / project ACCUMULATE:
 *     the caller zeroes them first.  This is what makes view chunking,
 *     checkpoint/resume (volume + next view index) and adjoint sums exact.
 *   - Errors: every call returns an ifdk_status (0 = success, negative =
 *     failure); argument errors are detected before any launch and leave all
 *     buffers untouched.  Nothing is thrown or printed.  Faults found on the
 *     device (a bounded wait that ran out) are latched in the plan's status
 *     word and reported by ifdk_last_device_status.
 *   - One plan is used by one host thread at a time.  Calls on one plan may be
 *     enqueued on any streams, with two exceptions that must not overlap on
 *     the device with another call of the same kind on the plan: packed
 *     back-projections that use the view split (they share the plan's partial
 *     volumes) and ifdk_backproject_host (it uses the plan's copy stream).
 */
#ifndef IFDK_H
#define IFDK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ifdk_plan_s *ifdk_plan;

/* Circular cone-beam geometry (Table 1).  Lengths in mm, angles in rad.
   `angles` (and `view_weights` if not NULL) are host arrays of np doubles,
   copied by ifdk_create. */
typedef struct {
    double sid, sdd;            /* d: source to rotation axis, D: source to detector */
    int nu, nv;                 /* detector width (U) and height (V), pixels */
    double du, dv;              /* detector pitch, mm/pixel */
    double off_u, off_v;        /* principal point offset from the detector centre, mm */
    int np;                     /* number of views */
    const double *angles;       /* np view angles (rad) */
    const double *view_weights; /* np angular weights (rad), or NULL: half the angular
                                   distance to the two neighbouring views (2 pi / np
                                   for a uniform full scan) */
    int nx, ny, nz;             /* volume size, voxels */
    double dx, dy, dz;          /* voxel pitch, mm/voxel */
    double vol_off_z;           /* world Z of the volume centre, mm */
} ifdk_geometry;

/* Storage types of filtered projections. */
enum { IFDK_F32 = 0, IFDK_F16 = 1, IFDK_BF16 = 2 };

/* Status codes. */
enum {
    IFDK_OK = 0,
    IFDK_ERR_INVALID = -1,      /* NULL pointer, bad size, range or enum */
    IFDK_ERR_GEOMETRY = -2,     /* geometry the method does not cover (e.g. a voxel
                                   behind the source plane, non-positive pitch) */
    IFDK_ERR_ALIGNMENT = -3,    /* a buffer is not 16-byte aligned */
    IFDK_ERR_CUDA = -4,         /* a CUDA runtime call failed (no device, launch error) */
    IFDK_ERR_TIMEOUT = -5,      /* a bounded device wait ran out (device status) */
    IFDK_ERR_NOMEM = -6,        /* ifdk_create could not allocate its tables */
    IFDK_ERR_UNSUPPORTED = -7,  /* valid request the library does not implement */
    IFDK_ERR_BOUNDS = -8        /* device status of a checked build (compiled with
                                   IFDK_CHECK): a kernel read outside its window */
};

/* Builds a plan: FP64 per-view projection terms P_s = (M1 . Mrot(b_s) . M0)[0:3]
   (Eq. 2) re-centred on the volume and principal point, the FDK view weights
   dbeta_s * d * D / (2 du), the cosine table F_cos (Table 1, Algorithm 1) and
   the Ram-Lak taps h(0)=1/4, h(odd n)=-1/(pi^2 n^2) (Kak & Slaney); everything
   is cast to FP32 and uploaded to the current CUDA device.  Validates the
   geometry (positive sizes and pitches, every voxel in front of the source).
   *out receives the plan, or NULL on failure.  Synchronous. */
int ifdk_create(ifdk_plan *out, const ifdk_geometry *g);

/* Releases a plan (device tables included).  NULL is accepted.  The caller
   makes sure no work using the plan is still in flight. */
int ifdk_destroy(ifdk_plan p);

/* Filtering stage, Algorithm 1: Q[s][v][n] = sum_m h(n-m) F_cos[v][m] E[s][v][m]
   for the np views: the cosine weight followed by an exact linear (zero-padded)
   Ram-Lak convolution of every detector row, computed as a dense Toeplitz
   product (the convolution theorem of Sec. 2.2.3 is not used).
   E: device FP32 [np][nv][nu], read only, 16-byte aligned.  Q: device
   [np][nv][nu] of q_dtype (IFDK_F32, IFDK_F16 or IFDK_BF16), overwritten,
   16-byte aligned.  E and Q must not overlap.
   split_terms = 1..3: tensor cores (tcgen05).  The convolution is summed by
   parts, Q = sum_k g(n-k) d(k) over k = 0..nu, with d the first difference of
   the weighted row and g the running sum of the taps (the same result, but
   without the ~1400x cancellation of the direct sum at 2048 pixels); BF16
   operands are split into terms and accumulated in FP32: 1 = one BF16
   product; 2 = 2 terms each, 3 products, for 16-bit storage; 3 = 3 terms
   each, 6 products, FP32-level accuracy.  It needs a device workspace of at
   least the minimum that
   ifdk_filter_workspace_size reports, 128-byte aligned, owned by the caller
   and not used by anything else until the call's work has run (larger
   workspaces process more rows per launch).  split_terms = 0: FP32 SIMT
   kernel of the same sum by parts, workspace ignored (may be NULL).
   With ifdk_set_short_scan on, E is also weighted by 2 w(beta_s, gamma_m)
   together with F_cos. */
int ifdk_filter(ifdk_plan p, const float *E, void *Q, int q_dtype, int split_terms,
                void *workspace, size_t workspace_bytes, void *stream);

/* ifdk_filter with the range check of 16-bit storage: also writes
   view_max[s] = max |Q[s][v][n]| over view s, taken on the FP32 values before
   the rounding to q_dtype.  Each row's maximum is reduced with warp shuffles
   in the filter's epilogue, then one atomic max per view and warp.  A value
   above 65504 means that FP16 storage of the view overflowed to infinity.
   It is NaN if a value of the view is NaN.  view_max: device FP32 [np],
   4-byte aligned, owned by the caller, overwritten; the call zeroes it on
   `stream` first.  Other arguments, the workspace and errors as ifdk_filter;
   view_max NULL returns IFDK_ERR_INVALID. */
int ifdk_filter_max(ifdk_plan p, const float *E, void *Q, int q_dtype, int split_terms,
                    void *workspace, size_t workspace_bytes, float *view_max, void *stream);

/* ifdk_filter on a range of views: Ev (device FP32 [view_count][nv][nu]) holds
   views [view_begin, view_begin + view_count) and Qv (device [view_count][nv][nu]
   of q_dtype) receives them filtered, the same values ifdk_filter gives those
   views (row by row the same arithmetic).  This is the filtering of one batch
   of the paper's pipeline (Sec. 4: projections are filtered in batches as they
   arrive and handed on to the back-projection).  Arguments, workspace,
   alignment and errors as ifdk_filter; a range outside [0, np) returns
   IFDK_ERR_INVALID, view_count = 0 does nothing. */
int ifdk_filter_views(ifdk_plan p, const float *Ev, void *Qv, int q_dtype, int split_terms, int view_begin,
                      int view_count, void *workspace, size_t workspace_bytes, void *stream);

/* Workspace of ifdk_filter for split_terms: the minimum (one 128-row tile of
   split operands) and a preferred size (every row in one launch, up to 1 GiB).
   Either pointer may be NULL.  0 bytes for split_terms = 0. */
int ifdk_filter_workspace_size(ifdk_plan p, int split_terms, size_t *min_bytes,
                               size_t *preferred_bytes);

/* ifdk_filter's tensor-core path for callers that cannot allocate device
   memory: the same computation and arguments as ifdk_filter with
   split_terms 1..3, but the split-operand workspace is a fixed 16 MiB device
   array inside the library instead of a caller buffer, and the call allocates
   nothing.  It serves callers that own no device allocator at all (a plain C
   program that only holds the E and Q buffers handed to it by a host
   application) and callers that must not allocate once they run, such as
   scanner pipelines that reserve all device memory at start-up and keep it
   fixed while reconstructing.  The iFDK paper has no counterpart to this
   call.
   Limit: the array must hold one 128-row tile of split operands,
   split_terms * 128 * ceil((nu + 1) / 64) * 64 * 2 bytes; larger requests
   return IFDK_ERR_UNSUPPORTED before any work (nu up to 21823 for 3 terms).  Rows are
   processed in launches of at most 16 MiB of operands, so it is slower than
   ifdk_filter with a large workspace.
   Every GPU that loads the library holds the 16 MiB until the process exits.
   The first call on a device looks up the array's device address (with that
   device current) and should come before any stream capture.  The address is
   kept for the life of the process: after cudaDeviceReset, or anything else
   that destroys and recreates the device's primary context, it is stale and
   this call must not be used again in that process.  All calls share
   the array and it keeps the previous call's contents (nothing in it has to
   start at zero: every row read is written first by the same call); calls
   whose work overlaps on the GPU (other streams, other host threads) race on
   it and must be serialised by the caller. */
int ifdk_filter_noalloc(ifdk_plan p, const float *E, void *Q, int q_dtype, int split_terms,
                        void *stream);

/* Adjoint of ifdk_filter for FP32 (the Toeplitz matrix is symmetric because h
   is even, and F_cos is diagonal): G_E[s][v][m] = F_cos[v][m] sum_n h(n-m) G_Q[s][v][n].
   G_Q, G_E: device FP32 [np][nv][nu]; G_E is overwritten.  With
   ifdk_set_short_scan on, G_E is also weighted by 2 w(beta_s, gamma_m). */
int ifdk_filter_adjoint(ifdk_plan p, const float *G_Q, float *G_E, void *stream);

/* Back-projection, Algorithm 4: for every voxel and view s in
   [view_begin, view_begin+view_count):
     vol[i][j][k] += w_s f^2 interp2(Q_s, u, v),  f = 1/z,
   with (x, y, z) = P_s (i, j, k, 1), u = x f, v = y f (Eq. 2); interp2 is the
   bilinear interpolation of Algorithm 3 with floor and zero outside the
   detector; w_s = dbeta_s d D / (2 du) is the FDK constant.  Voxel pairs
   (k, nz-1-k) share u, f and W (Theorems 1-3) when the volume is centred.
   Q: device [np][nv][nu] of q_dtype (the full view set; only the requested
   range is read), 16-byte aligned.  vol: device FP32, 16-byte aligned,
   ACCUMULATED into.  Q and vol must not overlap. */
int ifdk_backproject(ifdk_plan p, const void *Q, int q_dtype, int view_begin, int view_count,
                     float *vol, void *stream);

/* ifdk_backproject with a buffer that holds only the called views: Qv is
   device [view_count][nv][nu] of q_dtype, Qv[0] being view view_begin (the
   paper's column decomposition, Sec. 4, where each worker holds a subset of
   the views; also the staging chunks of ifdk_backproject_host).  Same
   result, arithmetic and alignment rules as ifdk_backproject. */
int ifdk_backproject_views(ifdk_plan p, const void *Qv, int q_dtype, int view_begin, int view_count,
                           float *vol, void *stream);

/* Packed views: the filtered views rearranged for the mirror-pair back-
   projection (Theorem 1 pairs voxel k with voxel nz-1-k, whose detector rows
   are mirror images about v_c: v_mirror = 2 v_c - v).  Available when the
   volume is centred on the source plane (vol_off_z = 0) and 2 v_c is an
   integer (v_c = (nv-1)/2 + off_v/dv); otherwise these calls return
   IFDK_ERR_UNSUPPORTED and ifdk_backproject serves every geometry.
   A packed view is [rows][row_elems][4] of q_dtype: element (i, e), for
   i in [0, rows) and e in [0, row_elems), is detector row r = r0 + i with
   r0 = min(0, 2 v_c - (nv - 1)) (rows = floor(v_c) + 3 - r0) and column
   c = e - 1 (row_elems = nu + 1 rounded up to even) and holds
     Q[r][c], Q[2 v_c - r][c], Q[r][c+1] - Q[r][c], Q[2 v_c - r][c+1] - Q[2 v_c - r][c],
   where Q reads 0 outside the detector; the differences are formed in FP32
   from the stored values and rounded once to q_dtype.  For IFDK_BF16 the
   element holds the right taps instead of the differences:
     Q[r][c], Q[2 v_c - r][c], Q[r][c+1], Q[2 v_c - r][c+1]
   (every value a stored value; the kernel interpolates along U with BF16
   weights 1 - du and du and FP32 sums).  That is about twice
   the bytes of a view of Q; one shared-memory load then gives a voxel pair
   both taps of a detector row, and interpolating along U is one FMA (two for
   BF16).
   ifdk_packed_size reports view_bytes (bytes of one packed view), rows and
   row_elems (any pointer may be NULL). */
int ifdk_packed_size(ifdk_plan p, int q_dtype, size_t *view_bytes, int *rows, int *row_elems);

/* Packs view_count views: Q device [view_count][nv][nu] of q_dtype ->
   Qp device [view_count][rows][row_elems][4] of q_dtype (ifdk_packed_size),
   both 16-byte aligned, not overlapping.  One memory-bound pass (each value
   of Q is read twice and written twice).  Asynchronous on `stream`. */
int ifdk_pack_views(ifdk_plan p, const void *Q, int q_dtype, int view_count, void *Qp, void *stream);

/* Back-projection (Algorithm 4, the same sum as ifdk_backproject) from packed
   views: Qp device [np][rows][row_elems][4] of q_dtype (all views packed,
   ifdk_pack_views), 16-byte aligned; views [view_begin, view_begin +
   view_count) are added into vol (device FP32 [nx][ny][nz], 16-byte
   aligned).  TMA stages windows of packed views in shared memory as they
   are used (a ring of stages paced by mbarriers).  With half-turn view
   pairing (ifdk_set_view_pairing) the views of the range that pair up are
   back-projected together.  The fast path for FDK: ifdk_filter,
   ifdk_pack_views, ifdk_backproject_packed. */
int ifdk_backproject_packed(ifdk_plan p, const void *Qp, int q_dtype, int view_begin, int view_count,
                            float *vol, void *stream);

/* Half-turn view pairing of ifdk_backproject_packed and of the packed
   streaming path of ifdk_backproject_host (on by default).  When the scan
   holds, for every view s < np/2, the view s + np/2 turned by exactly pi
   (checked in FP64 at ifdk_create, e.g. any uniform full scan with even np)
   and ny is even, voxel (X, Y, Z) in view s and voxel (-X, -Y, Z) in view
   s + np/2 project to the same detector point (u, v) with the same z (Eq. 2:
   Mrot(b + pi) = -Mrot(b) in the XY plane).  A thread then owns columns
   (i, j) and (nx-1-i, ny-1-j) and each evaluation of the coordinates of
   Algorithm 4 serves four voxels: (i, j, k), (i, j, nz-1-k),
   (nx-1-i, ny-1-j, k), (nx-1-i, ny-1-j, nz-1-k), of the two views.  Same
   sum, different FP32 rounding order.  (The paper's Sec. 3.2 cites this
   kind of rotational symmetry, after Zhao et al., and leaves it out because
   its pipeline receives views in scan order.)  Views of a call whose partner
   is outside the call's view range are back-projected singly.
   Quarter-turn view quads (enable = 2): when, in addition, view s + np/4 is
   view s turned by exactly pi/2 (np a multiple of 4) and the column grid is
   square (nx = ny, even, dx = dy), voxel (X, Y, Z) in view s and voxel
   (Y, -X, Z) in view s + np/4 share (u, v, z), i.e. column (i, j) and
   column (nx-1-j, i).  A thread then owns a column of one quadrant and its
   three images, and each evaluation of the coordinates serves eight voxels
   of the four views s, s + np/4, s + np/2, s + 3np/4 (the symmetry of Zhao
   et al. that Sec. 3.2 cites).  Quads serve a call over the whole scan
   (ifdk_backproject_packed and its pair-range form) and
   ifdk_backproject_packed_quads; other view ranges use pairs.
   enable = 0 turns pairing off for this plan, 1 selects half-turn pairs
   (the default), 2 quarter-turn quads where they apply (pairs elsewhere). */
int ifdk_set_view_pairing(ifdk_plan p, int enable);

/* ifdk_backproject_packed for the mirror pairs k in [pair_begin, pair_begin +
   pair_count) of the volume only (k < (nz+1)/2 pairs voxel k with nz-1-k): the
   paper's sub-volumes, a z-slab together with its mirror slab, which Theorem 1
   serves from the same view rows (Sec. 4 splits the volume into such pairs
   over the rows of its worker grid; each needs every view and no collective).
   vol: device FP32 [nx][ny][nz_out], 16-byte aligned, ACCUMULATED into, with
   nz_out = 2 pair_count (2 pair_count - 1 when nz is odd and the range holds
   the middle slice, which is its own mirror): voxel k of the volume is
   vol[..][k - pair_begin] and its mirror nz-1-k is vol[..][nz_out-1-(k - pair_begin)].
   Qp as for ifdk_backproject_packed (all np packed views).  The arithmetic per
   voxel is that of the whole-volume call.  Returns IFDK_ERR_INVALID for a
   range outside [0, (nz+1)/2). */
int ifdk_backproject_packed_pairs(ifdk_plan p, const void *Qp, int q_dtype, int view_begin, int view_count,
                                  int pair_begin, int pair_count, float *vol, void *stream);

/* Back-projection of one batch of half-turn view pairs (the paper's pipeline
   back-projects views in batches as they are filtered, Sec. 4): Qpb holds
   2 view_count packed views (ifdk_pack_views layout), first views
   [view_begin, view_begin + view_count), then their partners [view_begin +
   np/2, view_begin + np/2 + view_count); all of them are added into vol
   (device FP32 [nx][ny][nz], ACCUMULATED into).  With half-turn view pairing
   on and available the pairs are back-projected together (one launch),
   otherwise singly; either way the arithmetic per voxel is that of
   ifdk_backproject_packed over the same views.  np must be even and
   view_begin + view_count <= np/2 (else IFDK_ERR_INVALID).  Alignment and
   other errors as ifdk_backproject_packed. */
int ifdk_backproject_packed_batch(ifdk_plan p, const void *Qpb, int q_dtype, int view_begin, int view_count,
                                  float *vol, void *stream);

/* ifdk_backproject_packed_batch for quarter-turn view quads: Qpq holds
   4 view_count packed views, views [view_begin, view_begin + view_count) and
   then the same range shifted by np/4, np/2 and 3np/4 (ifdk_pack_views
   layout), all added into vol (device FP32 [nx][ny][nz], ACCUMULATED into).
   With quads on and available (ifdk_set_view_pairing mode 2) one launch
   serves them; otherwise half-turn pairs, or single views.  np must be a
   multiple of 4 and view_begin + view_count <= np/4 (else
   IFDK_ERR_INVALID).  Alignment and other errors as ifdk_backproject_packed. */
int ifdk_backproject_packed_quads(ifdk_plan p, const void *Qpq, int q_dtype, int view_begin, int view_count,
                                  float *vol, void *stream);

/* Describes a full-range ifdk_backproject_packed launch with q_dtype:
   info[0] = path (4 = quarter-turn view quads, 2 = half-turn view pairs,
   1 = single views, 0 = packed path not available), info[1] = TMA box width (elements), info[2] = box
   height (rows), info[3] = z pairs per thread, info[4] = TMA stages,
   info[5] = dynamic shared memory bytes per block, info[6] = blocks in the
   grid, info[7] = window width (pixels), info[8] = u alignment of the box
   start (pixels), info[9] = packed rows, info[10] = packed row elements,
   info[11] = r0, the detector row of packed row 0. */
int ifdk_backproject_packed_info(ifdk_plan p, int q_dtype, int64_t info[12]);

/* Host-only query (no device needed): ifdk_backproject_packed_info for this
   geometry and q_dtype with view pairing mode view_pairing (0, 1 or 2, as
   ifdk_set_view_pairing).  Returns the geometry's validation status. */
int ifdk_query_packed(const ifdk_geometry *g, int q_dtype, int view_pairing, int64_t info[12]);

/* Back-projection of filtered views streamed from host memory (the paper's
   Sec. 4 pipeline, where host-to-device transfer runs inside the
   back-projection time): views [view_begin, view_begin + view_count) are
   copied in chunks of chunk_views views into the two halves of `staging`
   on a copy stream owned by the plan and back-projected on `stream` as each
   chunk lands, so that the copy of chunk c+1 overlaps the back-projection
   of chunk c (two events per half order the reuse).
   Q_host: host array [np][host_nv][nu] of q_dtype whose rows
   [host_row0, host_row0 + nv) are the plan's detector rows (host_nv = nv,
   host_row0 = 0 when the host holds exactly the plan's detector; a plan
   built for the rows a slab reads, see ifdk_query_rows, streams only those
   rows out of full-height host views with one strided copy per chunk).
   It should be page-locked (cudaHostAlloc / cudaHostRegister), or the copies
   do not overlap.  staging: device, 256-byte aligned, at least
   2 * chunk_views * nv * nu * sizeof(q_dtype) bytes, owned by the caller.
   With packed views available (ifdk_packed_size) and staging of at least
   2 * chunk_views * (nv * nu * sizeof(q_dtype) + packed view_bytes) bytes,
   each chunk is packed on `stream` into the second part of the staging and
   back-projected by the kernels of ifdk_backproject_packed; with half-turn
   view pairing, the views that pair up travel first, in chunks of
   chunk_views / 2 views with their partners (two copies per chunk).
   Otherwise the kernels of ifdk_backproject read the chunks as copied.
   Asynchronous on `stream`: returns once everything is enqueued; Q_host,
   staging and vol must stay untouched until `stream` has passed this work.
   Copies start only after the work already on `stream`.  Calls on one plan
   must be issued from one host thread at a time and, when they overlap, on
   one stream (they share the plan's copy stream and events). */
int ifdk_backproject_host(ifdk_plan p, const void *Q_host, int q_dtype, int host_nv, int host_row0,
                          int view_begin, int view_count, int chunk_views, void *staging,
                          size_t staging_bytes, float *vol, void *stream);

/* Short scans (the scan variant beyond the Delta-beta rule).  A scan over
   pi + 2 delta with delta > the largest fan angle gamma measures some rays
   twice: (beta, gamma) again as (beta + pi + 2 gamma, -gamma).  enable = 1
   makes ifdk_filter, ifdk_filter_max, ifdk_filter_noalloc and
   ifdk_filter_adjoint also weight every projection by 2 w(beta_s, gamma_u)
   before the ramp filter.  w is Parker's weight (Med. Phys. 9, 1982), and a
   ray's two weights add to 1; the factor 2 replaces the 1/2 that the
   full-scan FDK constant holds for the double cover.  beta_s is measured from
   angles[0] and gamma_u = atan((u - u_c) Du / D).  The weights are formed in
   FP64 on the host and stored as FP32 [np][nu] in device memory owned by the
   plan.  The view weights stay those of ifdk_create; the first and last views
   get w = 0.  Returns IFDK_ERR_GEOMETRY unless the angles increase strictly
   over a range in (pi + 2 max|gamma|, 2 pi) with np >= 3; IFDK_ERR_NOMEM if
   the table cannot be allocated.  enable = 0 drops the weights.  Not safe to
   call while filter calls of the plan are in flight. */
int ifdk_set_short_scan(ifdk_plan p, int enable);

/* View split of the packed back-projection for small volumes.  Throughput
   falls as the volume shrinks against its input (the alpha of Table 5).
   A small volume has too few columns and z-runs to fill the GPU: its grid
   covers at most half a wave.  For such volumes (up to 64 MiB of partial
   volumes, allocated by ifdk_create) ifdk_backproject_packed splits the view
   range of each launch into S parts, one per grid layer.  S fills about one
   wave; each part holds at least 2 views or view pairs, and S <= 16.  Each
   part's sums are stored in a partial volume of the plan.  A second kernel
   then adds the parts to vol in part order, so results are reproducible but
   round differently from S = 1.  Launches that split share the plan's
   partial volumes: calls on one plan must not overlap on different streams
   while a split is in use.
   ifdk_set_view_split caps S: 0 = automatic (default), 1 = never split,
   n >= 2 = at most n.  Returns IFDK_ERR_INVALID for a negative cap.
   ifdk_view_split returns in *splits the S that a packed back-projection of
   all np views of q_dtype uses on this plan (1: no split). */
int ifdk_set_view_split(ifdk_plan p, int max_splits);
int ifdk_view_split(ifdk_plan p, int q_dtype, int *splits);

/* Exact adjoint of ifdk_backproject (FP32): for every voxel, view in the
   range and bilinear tap, P[s][tap] += w_s f^2 (bilinear weight) vol[i][j][k].
   It is the transpose of the back-projection matrix, not a physical line-
   integral projector.  vol: device FP32 [nx][ny][nz]; P: device FP32
   [np][nv][nu], ACCUMULATED into (floating-point atomics: the summation order,
   hence the last bits, may differ between runs). */
int ifdk_project(ifdk_plan p, const float *vol, float *P, int view_begin, int view_count,
                 void *stream);

/* Element-wise steps of the iterative solvers that reuse the back-projection
   and its adjoint (Sec. 1 and Sec. 6 name SART and MLEM as users of the
   back-projector): with A = ifdk_project and A^T the back-projection, one
   update over a subset S of the views is
     SART (Andersen & Kak 1984):  x <- x + lambda A_S^T((p - A x) / R) / C_S
     MLEM (Shepp & Vardi 1982; ordered subsets, Hudson & Larkin 1994):
                                  x <- x A_S^T(p / A x) / C_S
   with R = A 1 (ray sums over every voxel) and C_S = A_S^T 1 (voxel sums over
   the subset's rays).  A ray with R = 0 (SART) or A x = 0 (MLEM) gives 0; a
   voxel with C_S = 0 keeps its value.  The caller sequences the steps:
   ifdk_project of x over S's views into Ax (zeroed), ifdk_iter_ratio,
   a back-projection of the ratios into U (zeroed), ifdk_iter_update.
   ifdk_iter_ratio: Pm (measured views), Ax (A x), R (row sums; SART only,
   may be NULL for MLEM) and out are device FP32 arrays of view_count views
   [view_count][nv][nu] (pointers to the range's first view); out receives
   the ratio and Ax is set to 0 (ready for the next projection).
   ifdk_iter_update: x, U (the back-projected ratios) and C (C_S) are device
   FP32 [nx][ny][nz]; x is updated in place and U set to 0; nonneg = 1
   clips SART's x at 0 (ignored by MLEM, which keeps x >= 0 for p >= 0).
   Buffers 4-byte aligned (16-byte alignment takes the vector path), owned by
   the caller, not overlapping.  method: IFDK_SART or IFDK_MLEM.  One
   streaming pass each, asynchronous on `stream`. */
enum { IFDK_SART = 0, IFDK_MLEM = 1 };
int ifdk_iter_ratio(ifdk_plan p, int method, const float *Pm, float *Ax, const float *R, float *out,
                    int view_count, void *stream);
int ifdk_iter_update(ifdk_plan p, int method, float *x, float *U, const float *C, float lambda, int nonneg,
                     void *stream);

/* Output stage of Algorithm 4, I <- reshape(I~) (Sec. 3.3; the volume is
   stored as Nz slices of Nx x Ny, Sec. 4): writes slices [k_begin,
   k_begin + k_count) of the k-fastest volume vol (device FP32 [nx][ny][nz],
   as the back-projectors accumulate it) i-fastest into out (device
   [k_count][ny][nx] of out_dtype), i.e. out[k - k_begin][j][i] = vol[i][j][k].
   IFDK_F32 copies exactly; IFDK_F16 / IFDK_BF16 round to nearest even.
   Both buffers 16-byte aligned, owned by the caller, must not overlap; out
   is overwritten, vol is only read.  Range errors (k_begin < 0, k_count < 0,
   k_begin + k_count > nz) return IFDK_ERR_INVALID before any launch;
   k_count == 0 does nothing (the buffers may then be NULL).  Asynchronous
   on `stream`. */
int ifdk_volume_slices(ifdk_plan p, const float *vol, void *out, int out_dtype, int k_begin,
                       int k_count, void *stream);

/* Reads and clears the plan's device status word on `stream` (synchronises
   that stream).  Returns IFDK_OK, IFDK_ERR_TIMEOUT if a bounded wait inside a
   kernel ran out since the last call, or IFDK_ERR_CUDA. */
int ifdk_last_device_status(ifdk_plan p, void *stream);

/* Sets the limit of every bounded device wait launched with this plan, in
   nanoseconds (default 2e9).  0 restores the default. */
int ifdk_set_wait_limit(ifdk_plan p, uint64_t nanoseconds);

/* Self-test of the bounded-wait machinery: launches one block that waits on an
   mbarrier nothing arrives at, for at most `nanoseconds`, then records
   IFDK_ERR_TIMEOUT in the status word and exits cleanly.  Asynchronous. */
int ifdk_wait_selftest(ifdk_plan p, uint64_t nanoseconds, void *stream);

/* Test hook of the packed back-projection's timeout path (no device fault is
   involved): with group >= 0, every block of the following packed
   back-projections on this plan (ifdk_backproject_packed and its pair-range,
   batch and streaming forms) acts as if its bounded wait for view group
   `group` (counted from 0 within the block's views: the launch's views, or
   its share of them under the view split; two groups per half-turn pair)
   had run out: it records IFDK_ERR_TIMEOUT in the plan's status word, waits
   for the copies it issued that may still be landing in its shared memory,
   and leaves; blocks that start after that skip their work.  The volume's
   contents are then undefined.  group < 0 turns the hook off (the default).
   Returns IFDK_ERR_INVALID for a NULL plan. */
int ifdk_set_test_abort(ifdk_plan p, int group);

/* Describes the launch the plan chose for ifdk_backproject with q_dtype:
   info[0] = path (1 = mirror-pair fold kernel, 0 = general kernel),
   info[1] = TMA box width (pixels), info[2] = box height (rows),
   info[3] = z pairs per thread, info[4] = views per shared-memory chunk,
   info[5] = dynamic shared memory bytes per block, info[6] = blocks in the grid
   (per launch of at most info[7] views), info[7] = views per launch. */
int ifdk_backproject_info(ifdk_plan p, int q_dtype, int64_t info[8]);

/* Host-only query (no device needed): the launch ifdk_backproject would use
   for this geometry and q_dtype, in the layout of ifdk_backproject_info,
   plus info[8] = fold width (elements) and info[9] = u alignment of the box
   start (elements).  Returns the geometry's validation status. */
int ifdk_query_backproject(const ifdk_geometry *g, int q_dtype, int64_t info[10]);

/* Host-only query: the detector rows [*row_begin, *row_begin + *row_count)
   that back-projecting views [view_begin, view_begin + view_count) of this
   geometry can read, from FP64 bounds of v over the volume (v - v_c is
   (B2 k' + B3) / z with z affine in (i', j'), so its extremes sit at the
   corners; Eq. 3, Theorems 2-3), widened by one row on each side and clipped
   to the detector.  *row_count = 0 when no voxel projects onto the detector.
   A plan whose detector is cut to these rows (nv = *row_count and
   off_v shifted by ((nv_full - 1) / 2 - *row_begin - (*row_count - 1) / 2) * dv,
   so that v_c moves by -*row_begin) back-projects the same volume. */
int ifdk_query_rows(const ifdk_geometry *g, int view_begin, int view_count, int *row_begin,
                    int *row_count);

/* Arithmetic rate probe: the denominator of the back-projection's roofline.
   Algorithm 4 with Algorithm 3 costs about ten arithmetic operations per
   voxel-view update (GUPS, Sec. 2.3) and very few projection bytes, so its
   bound is an arithmetic issue rate.  This call launches `blocks` blocks of
   1024 threads (one per SM: pass the SM count), each thread running 8
   independent chains of `iters` * 16 instructions of one kind:
     IFDK_RATE_FFMA        fma.rn.f32        (1 FP32 lane operation)
     IFDK_RATE_FFMA2       fma.rn.f32x2      (2: packed FP32 pair)
     IFDK_RATE_HFMA2       fma.rn.f16x2      (2: packed FP16 pair)
     IFDK_RATE_FMA_F32_F16 fma.rn.f32.f16    (1: FP16 product, FP32 sum)
     IFDK_RATE_LOP3        lop3.b32          (1: integer logic)
     IFDK_RATE_FMA_F32_BF16 fma.rn.f32.bf16  (1: BF16 product, FP32 sum)
   Each block records its SM clock (clock64) before and after its loop and its
   SM id: clocks[3 b + 0..2] = start, end, smid (device int64 [3 * blocks],
   8-byte aligned).  sink: device FP32 [blocks * 1024], overwritten with the
   chains' results.  out[0] = instructions per thread, out[1] = lane
   operations per instruction (host).  Rate per SM = 1024 * out[0] * out[1]
   / (end - start), lane operations per SM clock; the loop's own counter
   instructions (under 3 %) make it a lower bound.  Asynchronous on `stream`.
   The paper has no counterpart. */
enum { IFDK_RATE_FFMA = 0, IFDK_RATE_FFMA2 = 1, IFDK_RATE_HFMA2 = 2, IFDK_RATE_FMA_F32_F16 = 3,
       IFDK_RATE_LOP3 = 4, IFDK_RATE_FMA_F32_BF16 = 5 };
int ifdk_arith_rate(int kind, int blocks, long long iters, float *sink, long long *clocks,
                    int64_t out[2], void *stream);

/* Human-readable text for a status code (static storage). */
const char *ifdk_status_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* IFDK_H */
