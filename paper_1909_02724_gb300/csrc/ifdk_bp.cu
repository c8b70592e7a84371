// Back-projection (Algorithm 4 of the iFDK paper) for sm_103a.
//
// Mirror-pair kernels (volume centred on the source plane, 2 v_c integral):
//   * a block owns a 16 x 16 tile of (i, j) columns and kPairs z pairs
//     (k, nz-1-k); each thread owns one column and its z-run of pairs;
//   * per view, the block's detector footprint is staged by TMA as two boxes:
//     rows [v0, v0+H) for the direct half and the mirrored rows (Theorem 1:
//     v_mirror = 2 v_c - v), in chunks of views, double buffered on mbarriers;
//     TMA's zero fill implements "taps outside the detector read 0";
//   * per (column, view) a thread forms z, f = 1/z, u, W_dis = w f^2 and the row
//     slope once (Algorithm 4, Theorems 2 and 3) and reuses them over its z-run;
//     the pair (k, nz-1-k) shares u, f, W_dis and the row fraction (Theorem 1);
//   * consecutive pairs step about one detector row (the magnification), so the
//     u-interpolated taps of a row are loaded once and reused by the next pair
//     whenever it starts on the row the previous one ended on;
//   * direct and mirror voxel run side by side in packed f32x2 arithmetic and
//     accumulate in FP32 registers over all views; the volume is written once
//     (read-modify-write, vectorised, 64-bit offsets, k-major layout).
//   FP32 storage reads the taps straight from the boxes (row pitch = 16 mod 32
//   floats, so lanes on adjacent rows do not share banks).  FP16 / BF16
//   storage first folds the two boxes into one array whose 8-byte element
//   (m, c) holds Q[m][c], Q[2vc-m][c], Q[m][c+1], Q[2vc-m][c+1], so one load
//   serves both voxels of a pair.  FP16 taps are u-interpolated in FP16
//   (packed half2) and widened once; BF16 taps are widened (a shift) first.
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
    int u0a, v0, v0m, off;   // box origins (u0a aligned), column of the window start in the box
};

struct BpArgs {
    float *vol;
    const ViewTerms *terms;
    unsigned int *status;
    unsigned long long wait_ns;
    int nx, ny, nz, tiles_x;
    int view_begin, view_count, q_view0;   // Q holds views from q_view0 on
    int box_w, box_h, fold_w, two_vc, views;
    float cx, cy, cz, uc, vc;
    uint32_t raw_box_bytes;    // one box, rounded up to 128 bytes
    uint32_t box_tx_bytes;     // one box, exact (TMA transaction count)
};

template <typename T> struct StoreT;
template <> struct StoreT<float> {
    static constexpr int ALIGN = 4;
    static constexpr CUtensorMapDataType TMA = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
};
template <> struct StoreT<__half> {
    static constexpr int ALIGN = 8;
    static constexpr CUtensorMapDataType TMA = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
};
template <> struct StoreT<__nv_bfloat16> {
    static constexpr int ALIGN = 8;
    static constexpr CUtensorMapDataType TMA = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
};

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ float lds_f32(uint32_t a)
{
    float r;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(r) : "r"(a));
    return r;
}
__device__ __forceinline__ float4 lds_f32x4(uint32_t a)
{
    float4 r;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(a));
    return r;
}
__device__ __forceinline__ int4 lds_i32x4(uint32_t a)
{
    int4 r;
    asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "r"(a));
    return r;
}
__device__ __forceinline__ uint2 lds_u32x2(uint32_t a)
{
    uint2 r;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "r"(a));
    return r;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t a)
{
    unsigned short r;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(r) : "r"(a));
    return r;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a)
{
    uint32_t r;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r) : "r"(a));
    return r;
}
__device__ __forceinline__ void sts_f32x4(uint32_t a, float4 v)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ void sts_i32x4(uint32_t a, int4 v)
{
    asm volatile("st.shared.v4.s32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ void sts_u32x2(uint32_t a, uint2 v)
{
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(a), "r"(v.x), "r"(v.y) : "memory");
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Packed FP32 helpers (f32x2): lerp(a, b, t) = a + t (b - a), each step rounded once.
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float2 t)
{
    const float2 m1 = make_float2(-1.0f, -1.0f);
    return __ffma2_rn(t, __ffma2_rn(a, m1, b), a);
}

// Shared-memory map (offsets from a 128-byte aligned base).
constexpr uint32_t kSmemBars = 0;       // mbarrier
constexpr uint32_t kSmemAbort = 16;     // abort flag
constexpr uint32_t kSmemViews = 64;     // 2 slots x kViews ViewSmem (512 bytes)
constexpr uint32_t kSmemRaw = 1024;     // one stage of views x 2 boxes, then 2 fold buffers

struct Block {
    int i0, j0, k0, i, j;
    float ip, jp, kp0;
};

__device__ __forceinline__ Block block_coords(const BpArgs &a)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // warp = 8 x 4 patch of columns, 2 x 4 warps per 16 x 16 tile
    const int tx = (warp & 1) * 8 + (lane & 7), ty = (warp >> 1) * 4 + (lane >> 3);
    Block b;
    b.i0 = (blockIdx.x % a.tiles_x) * kTileX;
    b.j0 = (blockIdx.x / a.tiles_x) * kTileY;
    b.k0 = blockIdx.y * kPairs;
    b.i = b.i0 + tx;
    b.j = b.j0 + ty;
    b.ip = (float)b.i - a.cx;
    b.jp = (float)b.j - a.cy;
    b.kp0 = (float)b.k0 - a.cz;
    return b;
}

// Warp 0: window geometry of the nvc views of a chunk (lane v -> view v),
// written to `slot`, then lane 0 issues the 2 boxes per view on `bar`.
template <int ALIGN>
__device__ __forceinline__ void stage_chunk(const BpArgs &a, const Block &b, const void *tmap, int first_view,
                                            int nvc, uint32_t slot, uint32_t raw_stage, uint32_t bar)
{
    const int lane = threadIdx.x & 31;
    if (lane < nvc) {
        const int s = first_view + lane;
        const float4 *tp = reinterpret_cast<const float4 *>(a.terms + s);
        const float4 t0 = __ldg(tp), t1 = __ldg(tp + 1), t2 = __ldg(tp + 2);
        // t0 = (A0, A1, A3, B2), t1 = (B3, C0, C1, C3), t2 = (w, -, -, -)
        const float ia = (float)b.i0 - a.cx, ib = ia + (kTileX - 1);
        const float ja = (float)b.j0 - a.cy, jb = ja + (kTileY - 1);
        float zc[4], uq[4];
        const float ci[4] = {ia, ib, ia, ib}, cj[4] = {ja, ja, jb, jb};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            zc[q] = fmaf(t1.y, ci[q], fmaf(t1.z, cj[q], t1.w));
            uq[q] = fmaf(t0.x, ci[q], fmaf(t0.y, cj[q], t0.z)) / zc[q];
        }
        const float u_lo = fminf(fminf(uq[0], uq[1]), fminf(uq[2], uq[3]));
        const float z_lo = fminf(fminf(zc[0], zc[1]), fminf(zc[2], zc[3]));
        const float z_hi = fmaxf(fmaxf(zc[0], zc[1]), fmaxf(zc[2], zc[3]));
        const float e0 = fmaf(t0.w, b.kp0, t1.x), e1 = fmaf(t0.w, b.kp0 + (kPairs - 1), t1.x);
        const float v_lo = fminf(fminf(e0 / z_lo, e0 / z_hi), fminf(e1 / z_lo, e1 / z_hi));
        const int u0f = (int)floorf(a.uc + u_lo) - kMargin;
        const int u0a = floor_div(u0f, ALIGN) * ALIGN;
        const int v0 = (int)floorf(a.vc + v_lo) - kMargin;
        const uint32_t d = slot + lane * (uint32_t)sizeof(ViewSmem);
        sts_f32x4(d, t0);
        sts_f32x4(d + 16, t1);
        sts_f32x4(d + 32, make_float4(t2.x, a.uc - (float)u0f, a.vc - (float)v0, 0.0f));
        sts_i32x4(d + 48, make_int4(u0a, v0, a.two_vc - v0 - a.box_h + 1, u0f - u0a));
    }
    __syncwarp();
    if (lane == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)nvc * 2u * a.box_tx_bytes);
        for (int v = 0; v < nvc; ++v) {
            const int4 o = lds_i32x4(slot + v * (uint32_t)sizeof(ViewSmem) + 48);
            const uint32_t dst = raw_stage + 2u * v * a.raw_box_bytes;
            tma_load_3d(dst, tmap, o.x, o.y, first_view + v - a.q_view0, bar);
            tma_load_3d(dst + a.raw_box_bytes, tmap, o.x, o.z, first_view + v - a.q_view0, bar);
        }
    }
}

// 1/z for z > 0 (here z >= 0.1 d): hardware approximation refined by one
// Newton-Raphson step r (2 - z r), within an ulp or so of the rounded quotient.
__device__ __forceinline__ float rcp_nr(float z)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(z));
    return r * fmaf(-z, r, 2.0f);
}

// Per (column, view) terms of Algorithm 4 (Theorems 2, 3).
struct ColView {
    float du, W, sig, vb;
    uint32_t tu;   // floor_frac bits of u - u_window
};

__device__ __forceinline__ ColView col_view(uint32_t vs, const Block &b)
{
    const float4 t0 = lds_f32x4(vs), t1 = lds_f32x4(vs + 16), t2 = lds_f32x4(vs + 32);
    ColView c;
    const float z = fmaf(t1.y, b.ip, fmaf(t1.z, b.jp, t1.w));
    const float f = rcp_nr(z);
    const float x = fmaf(t0.x, b.ip, fmaf(t0.y, b.jp, t0.z));
    const float ul = fmaf(x, f, t2.y);
    c.tu = floor_frac(ul, c.du);
    c.W = t2.x * f * f;
    c.sig = t0.w * f;
    c.vb = fmaf(c.sig, b.kp0, fmaf(t1.x, f, t2.z));
    return c;
}

// Writes the thread's z-run: acc[p].x -> voxel k0+p, acc[p].y -> its mirror nz-1-k0-p.
__device__ __forceinline__ void write_run(const BpArgs &a, const Block &b, const float2 *acc)
{
    constexpr int L = kPairs;
    static_assert(L % 4 == 0, "the vector path stores float4 runs from k0 = a multiple of L");
    if (b.i >= a.nx || b.j >= a.ny) return;
    float *col = a.vol + ((size_t)b.i * a.ny + b.j) * (size_t)a.nz;
    const int half = a.nz / 2, npairs = (a.nz + 1) / 2;
    if ((a.nz & 3) == 0 && b.k0 + L <= half) {
        float4 *pd = reinterpret_cast<float4 *>(col + b.k0);
        float4 *pm = reinterpret_cast<float4 *>(col + (a.nz - b.k0 - L));
#pragma unroll
        for (int q = 0; q < L / 4; ++q) {
            float4 d = pd[q];
            d.x += acc[4 * q].x; d.y += acc[4 * q + 1].x; d.z += acc[4 * q + 2].x; d.w += acc[4 * q + 3].x;
            pd[q] = d;
            float4 m = pm[q];   // voxels nz-k0-L+4q .. +3 mirror pairs L-1-4q .. L-4-4q
            m.x += acc[L - 1 - 4 * q].y; m.y += acc[L - 2 - 4 * q].y;
            m.z += acc[L - 3 - 4 * q].y; m.w += acc[L - 4 - 4 * q].y;
            pm[q] = m;
        }
    } else {
#pragma unroll
        for (int p = 0; p < L; ++p) {
            const int k = b.k0 + p;
            if (k < npairs) {
                col[k] += acc[p].x;
                const int km = a.nz - 1 - k;
                if (km > k) col[km] += acc[p].y;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Fold kernel (any storage type): the two boxes are folded into one array
// whose element (m, c) holds Q[m][c], Q[2vc-m][c], Q[m][c+1], Q[2vc-m][c+1]
// (direct and mirror row, two columns): one vector load per row serves both
// voxels of a pair.  Branch-free pair loop: two row loads per pair.
template <typename T> struct FoldElem;
template <> struct FoldElem<float> {
    static constexpr int ES = 16;
    // u-interpolated (direct, mirror) taps of one fold row
    __device__ __forceinline__ static float2 row(uint32_t a, float2 du2, __half2)
    {
        const float4 e = lds_f32x4(a);
        return lerp2(make_float2(e.x, e.y), make_float2(e.z, e.w), du2);
    }
};
template <> struct FoldElem<__half> {
    static constexpr int ES = 8;
    // the two stored FP16 taps are interpolated in FP16 (one packed sub + fma),
    // and the result is widened to FP32 once
    __device__ __forceinline__ static float2 row(uint32_t a, float2, __half2 duh)
    {
        const uint2 e = lds_u32x2(a);
        __half2 hx, hy;
        *reinterpret_cast<uint32_t *>(&hx) = e.x;
        *reinterpret_cast<uint32_t *>(&hy) = e.y;
        return __half22float2(__hfma2(duh, __hsub2(hy, hx), hx));
    }
};
template <> struct FoldElem<__nv_bfloat16> {
    static constexpr int ES = 8;
    __device__ __forceinline__ static float2 row(uint32_t a, float2 du2, __half2)
    {
        const uint2 e = lds_u32x2(a);
        return lerp2(make_float2(__uint_as_float(e.x << 16), __uint_as_float(e.x & 0xffff0000u)),
                     make_float2(__uint_as_float(e.y << 16), __uint_as_float(e.y & 0xffff0000u)), du2);
    }
};

template <typename T>
__device__ __forceinline__ float2 fold_row(uint32_t a, float2 du2, __half2 duh)
{
    return FoldElem<T>::row(a, du2, duh);
}

// The z-run of one (column, view): pair p samples rows n_p, n_p + 1 at
// v_p = vb + p sig (window coordinates).  With REUSE (every lane of the warp
// has sig < 1, so n_{p+1} - n_p is 0 or 1) each pair loads only row n_p + 1
// and takes row n_p from the previous pair's upper row when it moved up;
// otherwise both rows are loaded.  Both forms are branch-free.
template <typename T, int ES, uint32_t ROW, bool REUSE>
__device__ __forceinline__ void pair_loop(float2 *acc, uint32_t base, float sig, float vb, float2 du2, __half2 duh,
                                          float2 W2)
{
    constexpr int L = kPairs;
    float dv;
    uint32_t tv = floor_frac(vb, dv);
    uint32_t ad = base + tv * ROW;
    float2 lo = fold_row<T>(ad, du2, duh), hi = fold_row<T>(ad + ROW, du2, duh);
    acc[0] = __ffma2_rn(W2, lerp2(lo, hi, make_float2(dv, dv)), acc[0]);
#pragma unroll
    for (int p = 1; p < L; ++p) {
        const uint32_t tn = floor_frac(fmaf((float)p, sig, vb), dv);
        ad = base + tn * ROW;
        if constexpr (REUSE) {
            const bool moved = tn != tv;
            tv = tn;
            const float2 hn = fold_row<T>(ad + ROW, du2, duh);
            lo = moved ? hi : lo;
            hi = hn;
        } else {
            lo = fold_row<T>(ad, du2, duh);
            hi = fold_row<T>(ad + ROW, du2, duh);
        }
        acc[p] = __ffma2_rn(W2, lerp2(lo, hi, make_float2(dv, dv)), acc[p]);
    }
}

template <typename T, int FP>
__global__ void __launch_bounds__(kThreads, 3)
    bp_pairs_fold_kernel(const BpArgs a, const __grid_constant__ CUtensorMap tmap)
{
    constexpr int ES = FoldElem<T>::ES, ALIGN = StoreT<T>::ALIGN;
    constexpr uint32_t ROW = FP * ES;   // fold row pitch, bytes
    constexpr uint32_t VS = kViews * sizeof(ViewSmem);
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    const uint32_t sbase = smem_addr(smem_dyn);
    const uint32_t s0 = sbase + ((128u - (sbase & 127u)) & 127u);
    const uint32_t bar = s0 + kSmemBars, views0 = s0 + kSmemViews, raw = s0 + kSmemRaw;
    const int V = a.views, H = a.box_h, BW = a.box_w, FW = a.fold_w;
    const uint32_t fold0 = raw + 2u * V * a.raw_box_bytes;   // one raw stage, then two fold buffers
    const uint32_t fold_bytes = (uint32_t)V * H * ROW;
    const Block b = block_coords(a);
    const int tid = threadIdx.x, warp = tid >> 5;

    if (tid == 0) {
        prefetch_tmap(&tmap);
        mbar_init(bar, 1);
        sts_u32(s0 + kSmemAbort, 0u);
        fence_barrier_init();
    }
    __syncthreads();

    const int nchunks = (a.view_count + V - 1) / V;
    // chunk cn uses view slot cn & 1, the raw stage, and mbarrier phase cn
    auto stage = [&](int cn) {
        stage_chunk<ALIGN>(a, b, &tmap, a.view_begin + cn * V, min(V, a.view_count - cn * V),
                           views0 + (cn & 1) * VS, raw, bar);
    };
    // wait for chunk cn's boxes, then fold them into buffer cn & 1 (warp = row
    // group, lane = column: conflict-free loads and stores, no divisions)
    auto fold_chunk = [&](int cn) {
        if (!mbar_wait_bounded(bar, cn & 1, a.wait_ns)) sts_u32(s0 + kSmemAbort, 1u);
        const int nvc = min(V, a.view_count - cn * V);
        const uint32_t fbuf = fold0 + (cn & 1) * fold_bytes, vslot = views0 + (cn & 1) * VS;
        const int lane = tid & 31, rgrp = tid >> 5;
        for (int v = 0; v < nvc; ++v) {
            const int off = lds_i32x4(vslot + v * sizeof(ViewSmem) + 48).w;
            const uint32_t rdv = raw + 2u * v * a.raw_box_bytes, rmv = rdv + a.raw_box_bytes;
            const uint32_t fv = fbuf + (uint32_t)v * H * ROW;
            for (int m = rgrp; m < H; m += kThreads / 32) {
                const uint32_t rdm = rdv + (uint32_t)(m * BW + off) * sizeof(T);
                const uint32_t rmm = rmv + (uint32_t)((H - 1 - m) * BW + off) * sizeof(T);
                for (int cc = lane; cc < FW; cc += 32) {
                    const uint32_t rd = rdm + cc * sizeof(T), rm = rmm + cc * sizeof(T);
                    const uint32_t fa = fv + m * ROW + cc * ES;
                    if constexpr (sizeof(T) == 4) {
                        sts_f32x4(fa, make_float4(lds_f32(rd), lds_f32(rm), lds_f32(rd + 4), lds_f32(rm + 4)));
                    } else {
                        const uint32_t p0 = lds_u16(rd) | (lds_u16(rm) << 16);
                        const uint32_t p1 = lds_u16(rd + 2) | (lds_u16(rm + 2) << 16);
                        sts_u32x2(fa, make_uint2(p0, p1));
                    }
                }
            }
        }
    };

    if (warp == 0) stage(0);
    fold_chunk(0);
    __syncthreads();

    float2 acc[kPairs];
#pragma unroll
    for (int p = 0; p < kPairs; ++p) acc[p] = make_float2(0.0f, 0.0f);

    bool aborted = lds_u32(s0 + kSmemAbort) != 0;
    int c = 0;
    for (; c < nchunks && !aborted; ++c) {
        // the raw stage was folded in the previous iteration: refill it with chunk c+1
        if (warp == 0 && c + 1 < nchunks) stage(c + 1);
        const int nvc = min(V, a.view_count - c * V);
        const uint32_t vslot = views0 + (c & 1) * VS, fbuf = fold0 + (c & 1) * fold_bytes;
        for (int v = 0; v < nvc; ++v) {
            const ColView cv = col_view(vslot + v * sizeof(ViewSmem), b);
            // element (n, cu) = base + bits(t_v) * ROW, n = bits(t_v) - bias
            const uint32_t base = fbuf + (uint32_t)v * H * ROW + (cv.tu - kFloorBias) * ES - kFloorBias * ROW;
            const float2 du2 = make_float2(cv.du, cv.du), W2 = make_float2(cv.W, cv.W);
            const __half2 duh = __float2half2_rn(cv.du);
            // sig < 1 - 2^-10 keeps fp32 rounding of v_{p+1} - v_p below one row
            if (__all_sync(0xffffffffu, cv.sig < 0.9990234375f))
                pair_loop<T, ES, ROW, true>(acc, base, cv.sig, cv.vb, du2, duh, W2);
            else
                pair_loop<T, ES, ROW, false>(acc, base, cv.sig, cv.vb, du2, duh, W2);
        }
        if (c + 1 < nchunks) fold_chunk(c + 1);
        __syncthreads();
        aborted = lds_u32(s0 + kSmemAbort) != 0;
    }
    if (aborted) {
        // record the timeout; keep shared memory alive until the one copy that may
        // still be in flight (chunk c, issued before the failing wait) has landed
        if (tid == 0) {
            atomicOr(a.status, kStatusTimeout);
            if (c < nchunks) mbar_wait_bounded(bar, c & 1, a.wait_ns);
        }
        return;
    }
    write_run(a, b, acc);
}

// ---------------------------------------------------------------------------
// General kernel: one thread per column and kGenZ consecutive voxels.
struct GenArgs {
    float *vol;
    const void *Q;
    const ViewTerms *terms;
    int nx, ny, nz, nu, nv, tiles_x;
    int view_begin, view_count, q_view0;   // Q holds views from q_view0 on
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
        const T *Qs = Q + (size_t)(s - a.q_view0) * a.nv * a.nu;
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

// Host-side sizing of the pair kernels' TMA boxes: analytic FP64 bounds of
// the largest detector footprint of any block over any view.
BpLaunch size_pairs(const ifdk_plan_s *p, int q_dtype)
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
    const int need_w = b.fold_w + b.align;   // the window starts up to align-1 into the box
    b.box_h = (int)std::ceil(hv) + 2 * kMargin + 3;
    b.box_w = (need_w + b.align - 1) / b.align * b.align;
    b.pitch = b.fold_w <= kFoldPitchS - 1 ? kFoldPitchS : kFoldPitchL;
    if (b.fold_w > kFoldPitchL - 1 || b.box_w > 256 || b.box_h > 256) return b;
    const size_t box_bytes = ((size_t)b.box_w * b.box_h * es + 127) / 128 * 128;
    // the most views per chunk that keep three blocks (80 registers each) per SM
    const int fes = q_dtype == IFDK_F32 ? 16 : 8;
    for (b.views = kViews; b.views >= 1; --b.views) {
        b.smem = 128 + kSmemRaw + (size_t)b.views * 2 * box_bytes;      // one raw stage
        b.smem += 2 * (size_t)b.views * b.box_h * b.pitch * fes;        // two fold buffers
        if (b.smem <= 74 * 1024 || b.views == 1) break;   // three blocks per SM
    }
    if (b.smem > 220 * 1024 || (size_t)g.np * g.nv * g.nu * es >= ((size_t)1 << 40) || zblocks > 65535) return b;
    b.path = 1;
    return b;
}

template <typename T>
int launch_pairs(ifdk_plan_s *p, const BpLaunch &b, const void *Q, int view_begin, int view_count, int q_view0,
                 int q_views, float *vol, cudaStream_t stream)
{
    const ifdk_geometry &g = p->g;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return IFDK_ERR_CUDA;
    const int es = sizeof(T);
    CUtensorMap tmap;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nu, (cuuint64_t)g.nv, (cuuint64_t)q_views};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nu * es, (cuuint64_t)g.nu * g.nv * es};
    const cuuint32_t box[3] = {(cuuint32_t)b.box_w, (cuuint32_t)b.box_h, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&tmap, StoreT<T>::TMA, 3, const_cast<void *>(Q), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return IFDK_ERR_CUDA;
    BpArgs a;
    a.vol = vol;
    a.terms = p->d_terms;
    a.status = p->d_status;
    a.wait_ns = p->wait_ns;
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
    a.tiles_x = (g.nx + kTileX - 1) / kTileX;
    a.view_begin = view_begin;
    a.view_count = view_count;
    a.q_view0 = q_view0;
    a.box_w = b.box_w; a.box_h = b.box_h; a.fold_w = b.fold_w;
    a.two_vc = p->two_vc;
    a.views = b.views;
    a.cx = (float)((g.nx - 1) / 2.0); a.cy = (float)((g.ny - 1) / 2.0); a.cz = (float)((g.nz - 1) / 2.0);
    a.uc = (float)p->uc; a.vc = (float)p->vc;
    a.box_tx_bytes = (uint32_t)(b.box_w * b.box_h * es);
    a.raw_box_bytes = (a.box_tx_bytes + 127u) / 128u * 128u;
    void (*kern)(const BpArgs, const CUtensorMap);
    kern = b.pitch == kFoldPitchS ? bp_pairs_fold_kernel<T, kFoldPitchS> : bp_pairs_fold_kernel<T, kFoldPitchL>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.smem) != cudaSuccess)
        return IFDK_ERR_CUDA;
    kern<<<dim3(b.grid_x, b.grid_y), kThreads, b.smem, stream>>>(a, tmap);
    return cudaGetLastError() == cudaSuccess ? IFDK_OK : IFDK_ERR_CUDA;
}

template <typename T>
int launch_general(ifdk_plan_s *p, const void *Q, int view_begin, int view_count, int q_view0, float *vol,
                   cudaStream_t stream)
{
    const ifdk_geometry &g = p->g;
    GenArgs a;
    a.vol = vol; a.Q = Q; a.terms = p->d_terms;
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz; a.nu = g.nu; a.nv = g.nv;
    a.tiles_x = (g.nx + kTileX - 1) / kTileX;
    a.view_begin = view_begin; a.view_count = view_count; a.q_view0 = q_view0;
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
        p->bp[t] = size_pairs(p, t);
        if (!p->bp[t].path) {   // general kernel grid
            p->bp[t].grid_x = ((p->g.nx + kTileX - 1) / kTileX) * ((p->g.ny + kTileY - 1) / kTileY);
            p->bp[t].grid_y = (p->g.nz + kGenZ - 1) / kGenZ;
            p->bp[t].smem = 0;
        }
    }
}

int launch_backproject(ifdk_plan_s *p, const void *Q, int q_dtype, int view_begin, int view_count, int q_view0,
                       int q_views, float *vol, cudaStream_t stream)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    const BpLaunch &b = p->bp[q_dtype];
    if (b.path == 1) {
        switch (q_dtype) {
        case IFDK_F32: return launch_pairs<float>(p, b, Q, view_begin, view_count, q_view0, q_views, vol, stream);
        case IFDK_F16: return launch_pairs<__half>(p, b, Q, view_begin, view_count, q_view0, q_views, vol, stream);
        default: return launch_pairs<__nv_bfloat16>(p, b, Q, view_begin, view_count, q_view0, q_views, vol, stream);
        }
    }
    switch (q_dtype) {
    case IFDK_F32: return launch_general<float>(p, Q, view_begin, view_count, q_view0, vol, stream);
    case IFDK_F16: return launch_general<__half>(p, Q, view_begin, view_count, q_view0, vol, stream);
    default: return launch_general<__nv_bfloat16>(p, Q, view_begin, view_count, q_view0, vol, stream);
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
