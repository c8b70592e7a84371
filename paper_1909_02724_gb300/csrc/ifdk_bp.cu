// Back-projection (Algorithm 4 of the iFDK paper) for sm_103a.
//
// Fold kernel (volume centred on the source plane, 2 v_c integral):
//   * a block owns a 16 x 16 tile of (i, j) columns and kPairs z pairs
//     (k, nz-1-k); each thread owns one column and its z-run of pairs;
//   * per view, the block's detector footprint is staged by TMA as two boxes,
//     rows [v0, v0+H) (direct half) and the mirrored rows (Theorem 1:
//     v_mirror = 2 v_c - v), in chunks of kViews views, double buffered on
//     mbarriers; TMA's zero fill implements "taps outside the detector read 0";
//   * the two boxes are folded into one shared-memory array whose element
//     (m, c) holds Q[m][c], Q[2vc-m][c], Q[m][c+1], Q[2vc-m][c+1]: the direct
//     voxel's taps at row m and its mirror's taps at the mirrored row, so one
//     vector load serves both voxels of a pair, which share u, f and W_dis
//     (Theorems 2, 3) and the row fraction (Theorem 1);
//   * per (column, view) the thread forms z, f = 1/z, u, W_dis = w f^2 and the
//     row slope once (Algorithm 4, the gray terms) and reuses them over its
//     z-run; per pair it needs one FMA for v, one floor and the bilinear taps;
//   * the volume accumulates in FP32 registers over all views and is written
//     once with vectorised read-modify-write (k-major layout, 64-bit offsets).
// General kernel: any geometry (off-centre volume, fractional 2 v_c, large
//   footprints, unaligned rows): Algorithm 4 without the mirror, taps read
//   through the read-only cache with explicit bounds (zero outside).
#include <algorithm>
#include <cmath>

#include "ifdk_device.cuh"
#include "ifdk_internal.h"

namespace ifdk {
namespace {

struct ViewSmem {          // per view of a staged chunk (64 bytes)
    float A0, A1, A3, B2;
    float B3, C0, C1, C3;
    float w, uc_l, vc_l, pad;
    int u0a, v0, v0m, off;   // box origins (u0a aligned), fold column offset inside the box
};

struct FoldArgs {
    float *vol;
    const ViewTerms *terms;
    unsigned int *status;
    unsigned long long wait_ns;
    int nx, ny, nz, tiles_x;
    int view_begin, view_count;
    int box_w, box_h, fold_w, two_vc, views;
    float cx, cy, cz, uc, vc;
    uint32_t raw_box_bytes;    // one box, rounded up to 128 bytes
    uint32_t box_tx_bytes;     // one box, exact (TMA transaction count)
};

template <typename T> struct Fold;
template <> struct Fold<float> {            // element = 4 x f32
    static constexpr int ES = 16, ALIGN = 4;
    static constexpr CUtensorMapDataType TMA = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
};
template <> struct Fold<__half> {           // element = 4 x f16
    static constexpr int ES = 8, ALIGN = 8;
    static constexpr CUtensorMapDataType TMA = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
};
template <> struct Fold<__nv_bfloat16> {    // element = 4 x bf16
    static constexpr int ES = 8, ALIGN = 8;
    static constexpr CUtensorMapDataType TMA = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
};

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ float4 lds128(uint32_t a)
{
    float4 r;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "r"(a));
    return r;
}
__device__ __forceinline__ uint2 lds64(uint32_t a)
{
    uint2 r;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "r"(a));
    return r;
}

// Direct / mirror pair of a 2x2 tap block: (x = column c, y = column c+1).
struct Taps { float2 x, y; };

template <typename T> __device__ __forceinline__ Taps load_taps(uint32_t a);
template <> __device__ __forceinline__ Taps load_taps<float>(uint32_t a)
{
    const float4 e = lds128(a);
    return {make_float2(e.x, e.y), make_float2(e.z, e.w)};
}
template <> __device__ __forceinline__ Taps load_taps<__half>(uint32_t a)
{
    const uint2 e = lds64(a);
    __half2 hx, hy;
    *reinterpret_cast<uint32_t *>(&hx) = e.x;
    *reinterpret_cast<uint32_t *>(&hy) = e.y;
    return {__half22float2(hx), __half22float2(hy)};
}
template <> __device__ __forceinline__ Taps load_taps<__nv_bfloat16>(uint32_t a)
{
    const uint2 e = lds64(a);
    return {make_float2(__uint_as_float(e.x << 16), __uint_as_float(e.x & 0xffff0000u)),
            make_float2(__uint_as_float(e.y << 16), __uint_as_float(e.y & 0xffff0000u))};
}

// Shared-memory map of the fold kernel (offsets from a 128-byte aligned base).
constexpr uint32_t kSmemBars = 0;                 // 2 mbarriers
constexpr uint32_t kSmemViews = 64;               // 2 x kViews ViewSmem
constexpr uint32_t kSmemRaw = 1024;               // 2 stages x kViews x 2 boxes

template <typename T, int FP>
__global__ void __launch_bounds__(kThreads, 2)
    bp_fold_kernel(const FoldArgs a, const __grid_constant__ CUtensorMap tmap)
{
    constexpr int ES = Fold<T>::ES, ALIGN = Fold<T>::ALIGN;
    constexpr int L = kPairs;
    constexpr uint32_t ROW = FP * ES;              // fold row pitch (bytes)
    const int V = a.views;                         // views per chunk (<= kViews)
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~uintptr_t(127));
    ViewSmem *views = reinterpret_cast<ViewSmem *>(smem + kSmemViews);
    unsigned char *raw = smem + kSmemRaw;
    unsigned char *fold = raw + 2u * V * 2u * a.raw_box_bytes;
    const uint32_t bar0 = smem_addr(smem + kSmemBars);
    const int H = a.box_h, BW = a.box_w, FW = a.fold_w;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // warp = 8 x 4 patch of columns, 2 x 4 warps per 16 x 16 tile
    const int tx = (warp & 1) * 8 + (lane & 7), ty = (warp >> 1) * 4 + (lane >> 3);
    const int i0 = (blockIdx.x % a.tiles_x) * kTileX, j0 = (blockIdx.x / a.tiles_x) * kTileY;
    const int i = i0 + tx, j = j0 + ty;
    const int k0 = blockIdx.y * L;
    const float ip = (float)i - a.cx, jp = (float)j - a.cy;
    const float kp0 = (float)k0 - a.cz;

    if (tid == 0) {
        prefetch_tmap(&tmap);
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        fence_barrier_init();
    }
    __syncthreads();

    const int nchunks = (a.view_count + V - 1) / V;

    // Warp 0: geometry of chunk cn (lane v -> view v) and its TMA issue.
    auto stage_chunk = [&](int cn) {
        const int st = cn & 1;
        const int nvc = min(V, a.view_count - cn * V);
        if (lane < nvc) {
            const int s = a.view_begin + cn * V + lane;
            const float4 *tp = reinterpret_cast<const float4 *>(a.terms + s);
            const float4 t0 = __ldg(tp), t1 = __ldg(tp + 1), t2 = __ldg(tp + 2);
            // t0 = (A0, A1, A3, B2), t1 = (B3, C0, C1, C3), t2 = (w, -, -, -)
            const float ia = (float)i0 - a.cx, ib = ia + (kTileX - 1);
            const float ja = (float)j0 - a.cy, jb = ja + (kTileY - 1);
            float zc[4], uc[4];
            const float ci[4] = {ia, ib, ia, ib}, cj[4] = {ja, ja, jb, jb};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                zc[q] = fmaf(t1.y, ci[q], fmaf(t1.z, cj[q], t1.w));
                uc[q] = fmaf(t0.x, ci[q], fmaf(t0.y, cj[q], t0.z)) / zc[q];
            }
            const float u_lo = fminf(fminf(uc[0], uc[1]), fminf(uc[2], uc[3]));
            const float z_lo = fminf(fminf(zc[0], zc[1]), fminf(zc[2], zc[3]));
            const float z_hi = fmaxf(fmaxf(zc[0], zc[1]), fmaxf(zc[2], zc[3]));
            const float ka = kp0, kb = kp0 + (L - 1);
            const float e0 = fmaf(t0.w, ka, t1.x), e1 = fmaf(t0.w, kb, t1.x);
            const float v_lo = fminf(fminf(e0 / z_lo, e0 / z_hi), fminf(e1 / z_lo, e1 / z_hi));
            const int u0f = (int)floorf(a.uc + u_lo) - kMargin;
            const int u0a = floor_div(u0f, ALIGN) * ALIGN;
            const int v0 = (int)floorf(a.vc + v_lo) - kMargin;
            ViewSmem &vs = views[st * V + lane];
            vs.A0 = t0.x; vs.A1 = t0.y; vs.A3 = t0.z; vs.B2 = t0.w;
            vs.B3 = t1.x; vs.C0 = t1.y; vs.C1 = t1.z; vs.C3 = t1.w;
            vs.w = t2.x;
            vs.uc_l = a.uc - (float)u0f;
            vs.vc_l = a.vc - (float)v0;
            vs.pad = 0.0f;
            vs.u0a = u0a;
            vs.v0 = v0;
            vs.v0m = a.two_vc - v0 - H + 1;
            vs.off = u0f - u0a;
        }
        __syncwarp();
        if (lane == 0) {
            const uint32_t bar = bar0 + 8 * st;
            mbar_arrive_expect_tx(bar, (uint32_t)nvc * 2u * a.box_tx_bytes);
            for (int v = 0; v < nvc; ++v) {
                const ViewSmem &vs = views[st * V + v];
                const int s = a.view_begin + cn * V + v;
                const uint32_t dst = smem_addr(raw + ((st * V + v) * 2u) * a.raw_box_bytes);
                tma_load_3d(dst, &tmap, vs.u0a, vs.v0, s, bar);
                tma_load_3d(dst + a.raw_box_bytes, &tmap, vs.u0a, vs.v0m, s, bar);
            }
        }
    };

    if (warp == 0) stage_chunk(0);

    float2 acc[L];
#pragma unroll
    for (int p = 0; p < L; ++p) acc[p] = make_float2(0.0f, 0.0f);

    const int nseg = (FW + 7) / 8;
    bool failed = false;
    int c = 0;
    for (; c < nchunks; ++c) {
        const int st = c & 1;
        const int nvc = min(V, a.view_count - c * V);
        if (warp == 0 && c + 1 < nchunks) stage_chunk(c + 1);
        const bool ok = mbar_wait_bounded(bar0 + 8 * st, (c >> 1) & 1, a.wait_ns);
        if (__syncthreads_or(!ok)) { failed = true; break; }

        // Fold the raw boxes of this chunk: F[m][c] = (D[m][c], M[H-1-m][c], D[m][c+1], M[H-1-m][c+1]).
        for (int item = tid; item < nvc * H * nseg; item += kThreads) {
            const int v = item / (H * nseg), rem = item - v * (H * nseg);
            const int m = rem / nseg, seg = rem - m * nseg;
            const int off = views[st * V + v].off;
            const T *rd = reinterpret_cast<const T *>(raw + ((st * V + v) * 2u) * a.raw_box_bytes) + m * BW + off;
            const T *rm = reinterpret_cast<const T *>(raw + ((st * V + v) * 2u + 1u) * a.raw_box_bytes) +
                          (H - 1 - m) * BW + off;
            unsigned char *frow = fold + (size_t)(v * H + m) * ROW;
            const int cb = seg * 8, ce = min(FW, cb + 8);
            if constexpr (sizeof(T) == 4) {
                float d0 = rd[cb], m0 = rm[cb];
                for (int cc = cb; cc < ce; ++cc) {
                    const float d1 = rd[cc + 1], m1 = rm[cc + 1];
                    *reinterpret_cast<float4 *>(frow + cc * ES) = make_float4(d0, m0, d1, m1);
                    d0 = d1;
                    m0 = m1;
                }
            } else {
                const uint16_t *rd16 = reinterpret_cast<const uint16_t *>(rd);
                const uint16_t *rm16 = reinterpret_cast<const uint16_t *>(rm);
                uint32_t p0 = (uint32_t)rd16[cb] | ((uint32_t)rm16[cb] << 16);
                for (int cc = cb; cc < ce; ++cc) {
                    const uint32_t p1 = (uint32_t)rd16[cc + 1] | ((uint32_t)rm16[cc + 1] << 16);
                    *reinterpret_cast<uint2 *>(frow + cc * ES) = make_uint2(p0, p1);
                    p0 = p1;
                }
            }
        }
        __syncthreads();

        const uint32_t fold0 = smem_addr(fold);
        for (int v = 0; v < nvc; ++v) {
            const ViewSmem &vs = views[st * V + v];
            const float z = fmaf(vs.C0, ip, fmaf(vs.C1, jp, vs.C3));
            const float f = __frcp_rn(z);
            const float x = fmaf(vs.A0, ip, fmaf(vs.A1, jp, vs.A3));
            const float ul = fmaf(x, f, vs.uc_l);
            float du;
            const uint32_t tu = floor_frac(ul, du);
            const float W = vs.w * f * f;
            const float sig = vs.B2 * f;
            const float vb = fmaf(sig, kp0, fmaf(vs.B3, f, vs.vc_l));
            // address of fold element (n, cu) = base + bits(t_v) * ROW, n = bits(t_v) - 2^23 bias
            const uint32_t base = fold0 + (uint32_t)v * (uint32_t)H * ROW + (tu - kFloorBias) * ES -
                                  kFloorBias * ROW;
#pragma unroll
            for (int p = 0; p < L; ++p) {
                const float vl = fmaf((float)p, sig, vb);
                float dv;
                const uint32_t tv = floor_frac(vl, dv);
                const uint32_t ad = base + tv * ROW;
                const Taps lo = load_taps<T>(ad), hi = load_taps<T>(ad + ROW);
                const float lx = fmaf(du, lo.y.x - lo.x.x, lo.x.x);   // direct, row n
                const float ly = fmaf(du, lo.y.y - lo.x.y, lo.x.y);   // mirror, row 2vc-n
                const float hx = fmaf(du, hi.y.x - hi.x.x, hi.x.x);   // direct, row n+1
                const float hy = fmaf(du, hi.y.y - hi.x.y, hi.x.y);   // mirror, row 2vc-n-1
                acc[p].x = fmaf(W, fmaf(dv, hx - lx, lx), acc[p].x);
                acc[p].y = fmaf(W, fmaf(dv, hy - ly, ly), acc[p].y);
            }
        }
        __syncthreads();
    }

    if (failed) {
        // Record the timeout, then keep the block's shared memory alive until
        // every TMA copy it issued has landed (bounded again), and leave the
        // volume untouched.
        if (tid == 0) {
            atomicOr(a.status, kStatusTimeout);
            mbar_wait_bounded(bar0 + 8 * (c & 1), (c >> 1) & 1, a.wait_ns);
            if (c + 1 < nchunks)
                mbar_wait_bounded(bar0 + 8 * ((c + 1) & 1), ((c + 1) >> 1) & 1, a.wait_ns);
        }
        return;
    }

    if (i < a.nx && j < a.ny) {
        float *col = a.vol + ((size_t)i * a.ny + j) * (size_t)a.nz;
        const int half = a.nz / 2, npairs = (a.nz + 1) / 2;
        if ((a.nz & 3) == 0 && k0 + L <= half) {
            float4 *pd = reinterpret_cast<float4 *>(col + k0);
            float4 *pm = reinterpret_cast<float4 *>(col + (a.nz - k0 - L));
#pragma unroll
            for (int q = 0; q < L / 4; ++q) {
                float4 d = pd[q];
                d.x += acc[4 * q].x; d.y += acc[4 * q + 1].x; d.z += acc[4 * q + 2].x; d.w += acc[4 * q + 3].x;
                pd[q] = d;
                float4 m = pm[q];   // voxels nz-k0-L+4q .. +3 are mirrors of pairs L-1-4q .. L-4-4q
                m.x += acc[L - 1 - 4 * q].y; m.y += acc[L - 2 - 4 * q].y;
                m.z += acc[L - 3 - 4 * q].y; m.w += acc[L - 4 - 4 * q].y;
                pm[q] = m;
            }
        } else {
#pragma unroll
            for (int p = 0; p < L; ++p) {
                const int k = k0 + p;
                if (k < npairs) {
                    col[k] += acc[p].x;
                    const int km = a.nz - 1 - k;
                    if (km > k) col[km] += acc[p].y;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// General kernel: one thread per column and kGenZ consecutive voxels.
struct GenArgs {
    float *vol;
    const void *Q;
    const ViewTerms *terms;
    int nx, ny, nz, nu, nv, tiles_x;
    int view_begin, view_count;
    float cx, cy, cz, uc, vc;
};

template <typename T>
__device__ __forceinline__ float tap_at(const T *Qs, int nu, int nv, int iu, int iv)
{
    if ((unsigned)iu >= (unsigned)nu || (unsigned)iv >= (unsigned)nv) return 0.0f;
    return Storage<T>::to_float(Qs[(size_t)iv * nu + iu]);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) bp_general_kernel(const GenArgs a)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = (warp & 1) * 8 + (lane & 7), ty = (warp >> 1) * 4 + (lane >> 3);
    const int i = (blockIdx.x % a.tiles_x) * kTileX + tx, j = (blockIdx.x / a.tiles_x) * kTileY + ty;
    if (i >= a.nx || j >= a.ny) return;
    const int kb = blockIdx.y * kGenZ;
    const float ip = (float)i - a.cx, jp = (float)j - a.cy;
    float acc[kGenZ];
#pragma unroll
    for (int z = 0; z < kGenZ; ++z) acc[z] = 0.0f;
    const T *Q = static_cast<const T *>(a.Q);
    for (int s = a.view_begin; s < a.view_begin + a.view_count; ++s) {
        const float4 *tp = reinterpret_cast<const float4 *>(a.terms + s);
        const float4 t0 = __ldg(tp), t1 = __ldg(tp + 1), t2 = __ldg(tp + 2);
        const float z = fmaf(t1.y, ip, fmaf(t1.z, jp, t1.w));
        const float f = __frcp_rn(z);
        const float u = fmaf(fmaf(t0.x, ip, fmaf(t0.y, jp, t0.z)), f, a.uc);
        if (!(u > -2.0f && u < a.nu + 1.0f)) continue;
        const float fu = floorf(u);
        const int iu = (int)fu;
        const float du = u - fu;
        const float W = t2.x * f * f;
        const float sig = t0.w * f;
        const float vb = fmaf(t1.x, f, a.vc);
        const T *Qs = Q + (size_t)s * a.nv * a.nu;
#pragma unroll
        for (int zz = 0; zz < kGenZ; ++zz) {
            const float v = fmaf((float)(kb + zz) - a.cz, sig, vb);
            if (!(v > -2.0f && v < a.nv + 1.0f)) continue;
            const float fv = floorf(v);
            const int iv = (int)fv;
            const float dv = v - fv;
            const float q00 = tap_at(Qs, a.nu, a.nv, iu, iv), q01 = tap_at(Qs, a.nu, a.nv, iu + 1, iv);
            const float q10 = tap_at(Qs, a.nu, a.nv, iu, iv + 1), q11 = tap_at(Qs, a.nu, a.nv, iu + 1, iv + 1);
            const float t_lo = fmaf(du, q01 - q00, q00), t_hi = fmaf(du, q11 - q10, q10);
            acc[zz] = fmaf(W, fmaf(dv, t_hi - t_lo, t_lo), acc[zz]);
        }
    }
    float *col = a.vol + ((size_t)i * a.ny + j) * (size_t)a.nz;
#pragma unroll
    for (int zz = 0; zz < kGenZ; ++zz)
        if (kb + zz < a.nz) col[kb + zz] += acc[zz];
}

// Host-side sizing of the fold kernel's TMA boxes: analytic FP64 bounds of
// the largest detector footprint of any block over any view.
BpLaunch size_fold(const ifdk_plan_s *p, int q_dtype)
{
    const ifdk_geometry &g = p->g;
    BpLaunch b{};
    b.path = 0;
    const int es = (int)dtype_size(q_dtype);
    b.align = q_dtype == IFDK_F32 ? 4 : 8;
    const int tiles_x = (g.nx + kTileX - 1) / kTileX, tiles_y = (g.ny + kTileY - 1) / kTileY;
    const int npairs = (g.nz + 1) / 2, zblocks = (npairs + kPairs - 1) / kPairs;
    b.grid_x = tiles_x * tiles_y;
    b.grid_y = zblocks;
    if (!p->fold_ok || ((size_t)g.nu * es) % 16 != 0) return b;
    const double cx = (g.nx - 1) / 2.0, cy = (g.ny - 1) / 2.0, cz = (g.nz - 1) / 2.0;
    const double xa = cx * g.dx, xb = (tiles_x * kTileX - 1 - cx) * g.dx;
    const double ya = cy * g.dy, yb = (tiles_y * kTileY - 1 - cy) * g.dy;
    const double rxy = std::sqrt(std::max(xa * xa, xb * xb) + std::max(ya * ya, yb * yb));
    const double cmin = g.sid - rxy;
    if (cmin < 0.1 * g.sid) return b;
    const double et = std::hypot((kTileX - 1) * g.dx, (kTileY - 1) * g.dy);
    const double wu = g.sdd / g.du * et * (1.0 / cmin + 2.0 * rxy / (cmin * cmin));
    const double kmax = std::max(cz, (double)zblocks * kPairs - 1 - cz);
    const double b2 = g.sdd * g.dz / g.dv;
    const double hv = b2 * (kPairs - 1) / cmin + b2 * kmax * et / (cmin * cmin);
    b.fold_w = (int)std::ceil(wu) + 2 * kMargin + 2;
    b.box_w = ((b.fold_w + 1 + b.align - 1) + b.align - 1) / b.align * b.align;
    b.box_h = (int)std::ceil(hv) + 2 * kMargin + 3;
    b.pitch = b.fold_w <= kFoldPitchS - 1 ? kFoldPitchS : kFoldPitchL;
    const int fes = q_dtype == IFDK_F32 ? 16 : 8;
    const size_t box_bytes = ((size_t)b.box_w * b.box_h * es + 127) / 128 * 128;
    // the most views per chunk that keep two blocks per SM (else one)
    for (b.views = kViews; b.views >= 1; --b.views) {
        b.smem = 128 + kSmemRaw + 2 * b.views * 2 * box_bytes + (size_t)b.views * b.box_h * b.pitch * fes;
        if (b.smem <= 112 * 1024 || b.views == 1) break;
    }
    if (b.fold_w > kFoldPitchL - 1 || b.box_w > 256 || b.box_h > 256 || b.smem > 220 * 1024 ||
        (size_t)g.np * g.nv * g.nu * es >= ((size_t)1 << 40) || zblocks > 65535)
        return b;
    b.path = 1;
    return b;
}

template <typename T>
int launch_fold(ifdk_plan_s *p, const BpLaunch &b, const void *Q, int view_begin, int view_count,
                float *vol, cudaStream_t stream)
{
    const ifdk_geometry &g = p->g;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return IFDK_ERR_CUDA;
    const int es = sizeof(T);
    CUtensorMap tmap;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nu, (cuuint64_t)g.nv, (cuuint64_t)g.np};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nu * es, (cuuint64_t)g.nu * g.nv * es};
    const cuuint32_t box[3] = {(cuuint32_t)b.box_w, (cuuint32_t)b.box_h, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&tmap, Fold<T>::TMA, 3, const_cast<void *>(Q), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return IFDK_ERR_CUDA;
    FoldArgs a;
    a.vol = vol;
    a.terms = p->d_terms;
    a.status = p->d_status;
    a.wait_ns = p->wait_ns;
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
    a.tiles_x = (g.nx + kTileX - 1) / kTileX;
    a.view_begin = view_begin;
    a.view_count = view_count;
    a.box_w = b.box_w; a.box_h = b.box_h; a.fold_w = b.fold_w;
    a.two_vc = p->two_vc;
    a.views = b.views;
    a.cx = (float)((g.nx - 1) / 2.0); a.cy = (float)((g.ny - 1) / 2.0); a.cz = (float)((g.nz - 1) / 2.0);
    a.uc = (float)p->uc; a.vc = (float)p->vc;
    a.box_tx_bytes = (uint32_t)(b.box_w * b.box_h * es);
    a.raw_box_bytes = (a.box_tx_bytes + 127u) / 128u * 128u;
    auto kern = b.pitch == kFoldPitchS ? bp_fold_kernel<T, kFoldPitchS> : bp_fold_kernel<T, kFoldPitchL>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.smem) != cudaSuccess)
        return IFDK_ERR_CUDA;
    kern<<<dim3(b.grid_x, b.grid_y), kThreads, b.smem, stream>>>(a, tmap);
    return cudaGetLastError() == cudaSuccess ? IFDK_OK : IFDK_ERR_CUDA;
}

template <typename T>
int launch_general(ifdk_plan_s *p, const void *Q, int view_begin, int view_count, float *vol,
                   cudaStream_t stream)
{
    const ifdk_geometry &g = p->g;
    GenArgs a;
    a.vol = vol; a.Q = Q; a.terms = p->d_terms;
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.nu = g.nu; a.nv = g.nv;
    a.tiles_x = (g.nx + kTileX - 1) / kTileX;
    a.view_begin = view_begin; a.view_count = view_count;
    a.cx = (float)((g.nx - 1) / 2.0); a.cy = (float)((g.ny - 1) / 2.0); a.cz = (float)((g.nz - 1) / 2.0);
    a.uc = (float)p->uc; a.vc = (float)p->vc;
    const int tiles_y = (g.ny + kTileY - 1) / kTileY;
    const int zb = (g.nz + kGenZ - 1) / kGenZ;
    if (zb > 65535) return IFDK_ERR_UNSUPPORTED;
    bp_general_kernel<T><<<dim3(a.tiles_x * tiles_y, zb), kThreads, 0, stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? IFDK_OK : IFDK_ERR_CUDA;
}

}  // namespace

void plan_backproject(ifdk_plan_s *p)
{
    for (int t = 0; t < 3; ++t) {
        p->bp[t] = size_fold(p, t);
        if (!p->bp[t].path) {   // general kernel grid
            p->bp[t].grid_x = ((p->g.nx + kTileX - 1) / kTileX) * ((p->g.ny + kTileY - 1) / kTileY);
            p->bp[t].grid_y = (p->g.nz + kGenZ - 1) / kGenZ;
            p->bp[t].smem = 0;
        }
    }
}

int launch_backproject(ifdk_plan_s *p, const void *Q, int q_dtype, int view_begin, int view_count,
                       float *vol, cudaStream_t stream)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    const BpLaunch &b = p->bp[q_dtype];
    if (b.path == 1) {
        switch (q_dtype) {
        case IFDK_F32: return launch_fold<float>(p, b, Q, view_begin, view_count, vol, stream);
        case IFDK_F16: return launch_fold<__half>(p, b, Q, view_begin, view_count, vol, stream);
        default: return launch_fold<__nv_bfloat16>(p, b, Q, view_begin, view_count, vol, stream);
        }
    }
    switch (q_dtype) {
    case IFDK_F32: return launch_general<float>(p, Q, view_begin, view_count, vol, stream);
    case IFDK_F16: return launch_general<__half>(p, Q, view_begin, view_count, vol, stream);
    default: return launch_general<__nv_bfloat16>(p, Q, view_begin, view_count, vol, stream);
    }
}

// Bounded-wait self-test: waits on an mbarrier that nothing arrives at.
__global__ void wait_selftest_kernel(unsigned int *status, unsigned long long ns)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(b, 0, ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

int launch_wait_selftest(ifdk_plan_s *p, unsigned long long ns, cudaStream_t stream)
{
    wait_selftest_kernel<<<1, 32, 0, stream>>>(p->d_status, ns);
    return cudaGetLastError() == cudaSuccess ? IFDK_OK : IFDK_ERR_CUDA;
}

}  // namespace ifdk
