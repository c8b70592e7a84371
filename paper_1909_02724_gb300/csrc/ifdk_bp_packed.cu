// Back-projection (Algorithm 4 of the iFDK paper) from packed views, sm_103a.
//
// Packed views.  For a volume centred on the source plane with 2 v_c
// integral, voxel k and its mirror nz-1-k read detector rows that are mirror
// images about v_c (Theorem 1: v_mirror = 2 v_c - v).  A packed view stores
// for row r in [r0, floor(v_c) + 3), r0 = min(0, 2 v_c - (nv - 1)) (rows
// whose mirror lies on the detector), and column c in [-1, nu) the element
//   (Q[r][c], Q[2vc-r][c], Q[r][c+1] - Q[r][c], Q[2vc-r][c+1] - Q[2vc-r][c])
// (Q read as zero where a row or column lies outside the detector; column -1
// carries the first column as its right tap), so one shared-memory
// load gives both voxels of a pair the two taps of a detector row, and the
// interpolation along u is one FMA per pair (the difference is formed in
// FP32 when packing, then stored in the storage type).  BF16 storage keeps
// the right taps themselves, (Q[r][c], Q[2vc-r][c], Q[r][c+1], Q[2vc-r][c+1]):
// every value is a stored value, exact, and the interpolation along u is two
// FP32 FMAs of BF16 inputs per voxel.  Packing
// is one pass over Q (ifdk_pack_views); the back-projection then stages
// windows of packed views with TMA and uses them as they land.
//
// Kernel:
//   * a block owns a 16 x 16 tile of (i, j) columns and L z pairs
//     (k, nz-1-k); each thread owns one column and its z-run of pairs;
//   * per (column, view) a thread forms z, f = 1/z, u, W_dis = w f^2 and the
//     row slope once (Algorithm 4, Theorems 2 and 3) and reuses them over its
//     z-run; the pair (k, nz-1-k) shares u, f, W_dis and the row fraction;
//   * half-turn view pairs (NV = 2): when view s + P (P = np/2) is view s
//     turned by pi, voxel (X, Y, Z) in view s and voxel (-X, -Y, Z) in view
//     s + P have the same (u, v, z).  A thread owns column (i, j), j < ny/2,
//     and the opposite column (nx-1-i, ny-1-j).  Its coordinates in view s
//     serve its column with view s and the opposite column with view s + P;
//     its coordinates in view s + P serve its column with view s + P and the
//     opposite column with view s.  So each pair of views is two view groups,
//     and each evaluation of the coordinates, the row index and the row
//     fraction serves four voxel updates;
//   * quarter-turn view quads (NV = 4, FP16 storage): when view s + np/4 is
//     view s turned by pi/2 and the column grid is square, column (i, j) in
//     view s and column (nx-1-j, i) in view s + np/4 share (u, v, z).  A
//     thread owns a column of one quadrant and its three images under the
//     quarter turn; a view quad (s, s + np/4, s + np/2, s + 3np/4) is four
//     view groups, and each evaluation of the coordinates serves eight voxel
//     updates (the symmetry after Zhao et al. that Sec. 3.2 cites);
//   * a view group's window (the tile's detector footprint in the group's
//     own view, rows [v0, v0+H)) is one TMA box of the NV packed views of
//     the group's pair or quad together (a 4-D tensor map whose second
//     dimension steps from view s to view s + np/NV), so the views' elements
//     of a row sit side by side; TMA's zero fill implements "taps outside
//     the detector read 0";
//   * L2 locality: blocks take their column tiles in bands of 16 tile rows,
//     and each block starts its cycle over the views at a view group fixed by
//     its place in the launch order, so that the blocks resident at one time
//     work on the same views of a compact patch of columns and share the
//     windows in L2 (the views' order in a block's sum is fixed: the result
//     is reproducible);
//   * a ring of stages (one group each) paced by mbarriers: full = the box
//     landed, empty = every warp finished the group.  At group t, warp
//     t mod 8 refills the stage group t - 2 used with group t - 2 + stages
//     (the refill's latency, a wait and a few dependent loads, rotates over
//     the warps), so up to stages - 1 groups are in flight and warps never
//     meet at a block-wide barrier;
//   * consecutive pairs step about one detector row (the magnification), so
//     a pair loads only its upper row and takes the lower one from the
//     previous pair (after a step of two rows, it loads both);
//   * FP32 accumulation in registers over all views, one read-modify-write of
//     each thread's z-runs at the end (vectorised, 64-bit offsets, k-major).
//   FP32 storage: taps are interpolated in packed f32x2 arithmetic; BF16
//   storage: the u-lerp is (1 - du) Q_c + du Q_{c+1} as two FP32 FMAs of
//   BF16 inputs (fma.rn.f32.bf16: the weights rounded to BF16, products
//   exact, FP32 sum), so the taps are never widened, then the v-lerp and
//   accumulate in f32x2; FP16 storage: both lerps in packed half2, widened
//   once before the FP32 accumulate.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "ifdk_device.cuh"
#include "ifdk_internal.h"

namespace ifdk {
namespace {

constexpr int kPkMargin = 1;   // window margin (pixels) on every side
constexpr int kPkSwizzle = 16; // tile rows per band of the block order

struct PkGeom {              // per stage: the group's window and terms (64 bytes)
    float A0, A1, A3, B2;    // own view's projection terms (Eq. 2, re-centred)
    float B3, C0, C1, C3;
    float w0, uc_l, vc_l, w1;   // FDK weights of the box's view 0 / view 1; window-relative principal point
    int u0a, v0, pad0, pad1;    // box origin: column (element), row
};

struct PkArgs {
    float *vol;
    const ViewTerms *terms;
    unsigned int *status;
    unsigned long long wait_ns;
    int nx, ny, nz, tiles_x, ny_cols;   // ny_cols: rows j the grid covers (ny, or ny / 2 with NV = 2, 4)
    int nx_cols;                        // columns i the grid covers (nx, or nx / 2 with NV = 4)
    int view_begin, view_count;         // NV = 1: views; NV = 2: pairs (s, s + P), s from view_begin
    int q_view0, q_pair_off;            // view s is packed view s - q_view0 (its partner + q_pair_off)
    int pair_view_off;                  // view offset between the box's slots: np / NV
    int box_h, stages, row0;            // row0: detector row of packed row 0
    float cx, cy, cz, uc, vc;
    float wscale, wunscale;             // power of two on the FDK weights (FP16: keeps W in range) and its inverse
    uint32_t stage_bytes, box_tx_bytes;
    // view split (small volumes): block z takes part z of the view range and writes
    // (not adds) its sums to part + z * part_stride; nullptr: one part, added to vol
    float *part;
    size_t part_stride;
    int splits;
    int zfull;                          // z-blocks of L pairs; the rest take kPkTailL pairs
    // mirror pairs [pair0, pair_end) of the volume go to an output column of nz_out
    // voxels: the direct slab first (k - pair0), then its mirror (the whole volume:
    // pair0 = 0, pair_end = (nz + 1) / 2, nz_out = nz)
    int pair0, pair_end, nz_out;
    // test hook (ifdk_set_test_abort): every block treats its wait for view group
    // abort_group as expired (-1: off)
    int abort_group;
    int tiles_y;                        // column tiles along j the grid covers
    int resident;                       // blocks resident on the GPU at once (SMs x blocks per SM)
};

// Bound of the wait an aborting warp spends on the copies it issued that may
// still be landing in its shared memory: fixed, and independent of the plan's
// wait limit (which may be short, and has just run out), so that no block
// leaves while a bulk copy it started can still write to its shared memory.
constexpr unsigned long long kPkDrainNs = 2000000000ull;

template <typename T> struct PkT;
template <> struct PkT<float> {
    static constexpr int CODE = IFDK_F32;
    static constexpr int ALIGN = 1;
    static constexpr CUtensorMapDataType TMA = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
};
template <> struct PkT<__half> {
    static constexpr int CODE = IFDK_F16;
    static constexpr int ALIGN = 2;
    static constexpr CUtensorMapDataType TMA = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
};
template <> struct PkT<__nv_bfloat16> {
    static constexpr int CODE = IFDK_BF16;
    static constexpr int ALIGN = 2;
    static constexpr CUtensorMapDataType TMA = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
};

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ void sts_f32x4(uint32_t a, float4 v)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lds_u32_v(uint32_t a)
{
    uint32_t r;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r) : "r"(a));
    return r;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Orders this thread's earlier generic-proxy shared-memory accesses (and those
// it synchronised with) before its later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait for phase `parity`: spins on try_wait (which suspends the warp
// for a while in hardware) and reads the clock only every 16 tries.
__device__ __forceinline__ bool mbar_wait_lim(uint32_t bar, uint32_t parity, unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15u) == 0 && global_timer_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void *tmap, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Packed FP32 lerp(a, b, t) = a + t (b - a), each step rounded once.
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float2 t)
{
    const float2 m1 = make_float2(-1.0f, -1.0f);
    return __ffma2_rn(t, __ffma2_rn(a, m1, b), a);
}

// 1/z for z > 0 (here z >= 0.1 d): hardware approximation refined by one
// Newton-Raphson step r (2 - z r), within an ulp or so of the rounded quotient.
__device__ __forceinline__ float rcp_nr(float z)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(z));
    return r * fmaf(-z, r, 2.0f);
}

// Storage-type specific parts: element size, the u fraction as the row
// interpolation takes it (Du), the u-interpolated (direct, mirror) row of an
// element and the v-lerp + weighted accumulate of a pair.
template <typename T> struct Tap;
template <> struct Tap<float> {
    static constexpr uint32_t ES = 16;
    using R = float2;
    using Wt = float2;   // the weight of a pair, as the accumulate takes it
    using Du = float2;
    __device__ __forceinline__ static Wt weight(float w) { return make_float2(w, w); }
    __device__ __forceinline__ static Du frac_u(float du) { return make_float2(du, du); }
    __device__ __forceinline__ static R row(const unsigned char *e, Du du2)
    {
        const float4 q = *reinterpret_cast<const float4 *>(e);   // (taps at c, differences to c + 1)
        return __ffma2_rn(du2, make_float2(q.z, q.w), make_float2(q.x, q.y));
    }
    __device__ __forceinline__ static float2 accum(float2 acc, R lo, R hi, float2 dv2, __half2, Wt W2)
    {
        return __ffma2_rn(W2, lerp2(lo, hi, dv2), acc);
    }
};
template <> struct Tap<__half> {
    static constexpr uint32_t ES = 8;
    using R = __half2;
    // FP16 weight (the plan scales w by a power of two that keeps W in range)
    // for the mixed-precision accumulate below
    using Wt = unsigned short;
    using Du = __half2;
    __device__ __forceinline__ static Wt weight(float w) { return __half_as_ushort(__float2half_rn(w)); }
    __device__ __forceinline__ static Du frac_u(float du) { return __float2half2_rn(du); }
    __device__ __forceinline__ static R row(const unsigned char *e, Du duh)
    {
        const uint2 q = *reinterpret_cast<const uint2 *>(e);
        const __half2 hx = *reinterpret_cast<const __half2 *>(&q.x), hd = *reinterpret_cast<const __half2 *>(&q.y);
        return __hfma2(duh, hd, hx);
    }
    // v-lerp in half2, then acc += W r with FP16 inputs and FP32 accumulation,
    // one rounding (fma.rn.f32.f16)
    __device__ __forceinline__ static float2 accum(float2 acc, R lo, R hi, float2, __half2 dvh, Wt Wh)
    {
        const __half2 r = __hfma2(dvh, __hsub2(hi, lo), lo);
        const uint32_t rb = *reinterpret_cast<const uint32_t *>(&r);
        asm("{\n\t.reg .f16 rl, rh;\n\t"
            "mov.b32 {rl, rh}, %2;\n\t"
            "fma.rn.f32.f16 %0, %3, rl, %0;\n\t"
            "fma.rn.f32.f16 %1, %3, rh, %1;\n\t}"
            : "+f"(acc.x), "+f"(acc.y)
            : "r"(rb), "h"(Wh));
        return acc;
    }
};
template <> struct Tap<__nv_bfloat16> {
    static constexpr uint32_t ES = 8;
    using R = float2;
    using Wt = float2;
    using Du = uint32_t;   // the u weights (1 - du, du), each rounded to BF16 (low, high half)
    __device__ __forceinline__ static Wt weight(float w) { return make_float2(w, w); }
    __device__ __forceinline__ static Du frac_u(float du)
    {
        return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(1.0f - du)) |
               ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(du)) << 16);
    }
    // element (Q_c direct, Q_c mirror | Q_{c+1} direct, Q_{c+1} mirror): per voxel
    // du Q_{c+1} (exact: a product of two BF16 values fits FP32), then
    // + (1 - du) Q_c with one rounding
    __device__ __forceinline__ static R row(const unsigned char *e, Du wu)
    {
        const uint2 q = *reinterpret_cast<const uint2 *>(e);
        float2 r;
        asm("{\n\t.reg .b16 a0, a1, b0, b1, w0, w1;\n\t.reg .f32 z;\n\t"
            "mov.b32 {a0, a1}, %2;\n\t"
            "mov.b32 {b0, b1}, %3;\n\t"
            "mov.b32 {w0, w1}, %4;\n\t"
            "mov.f32 z, 0f00000000;\n\t"
            "fma.rn.f32.bf16 %0, w1, b0, z;\n\t"
            "fma.rn.f32.bf16 %1, w1, b1, z;\n\t"
            "fma.rn.f32.bf16 %0, w0, a0, %0;\n\t"
            "fma.rn.f32.bf16 %1, w0, a1, %1;\n\t}"
            : "=f"(r.x), "=f"(r.y)
            : "r"(q.x), "r"(q.y), "r"(wu));
        return r;
    }
    __device__ __forceinline__ static float2 accum(float2 acc, R lo, R hi, float2 dv2, __half2, Wt W2)
    {
        return __ffma2_rn(W2, lerp2(lo, hi, dv2), acc);
    }
};

// The z-run of one (column, view group): pair p samples box rows n_p, n_p + 1
// at v_p = vb + p sig (window coordinates).  The box holds NV views side by
// side in each row (rows ROWB bytes apart); the thread's column n reads the
// view that feeds it at shared offset cb[n] + row * ROWB (cb[n] = the element's
// offset in that view's slot) and accumulates it with weight W[n] into
// acc[n].  Row reuse by the
// warp's largest step (every lane votes): STEP1 (all sig < 1: n_{p+1} - n_p
// is 0 or 1) loads only row n_p + 1 and takes row n_p from the previous
// pair; STEP2 (sig < 2, which the plan guarantees: steps 0, 1 or 2) does the
// same and loads row n_p as well only after a step of 2 (a predicated load:
// less shared-memory traffic, for FP32 taps); ANY loads both rows.
enum class Reuse { STEP1, STEP2, ANY };

// Checked build (-DIFDK_CHECK): every tap read is tested against the stage's box;
// a read outside it sets kStatusBounds in the plan's status word and reads the
// box's first element instead.  Without the flag the macros add nothing.
#ifdef IFDK_CHECK
struct ChkBox {
    const unsigned char *lo, *hi;
    unsigned int *status;
};
template <typename T>
__device__ __forceinline__ const unsigned char *chk_row(const unsigned char *e, const ChkBox &c)
{
    if (e < c.lo || e + Tap<T>::ES > c.hi) {
        atomicOr(c.status, kStatusBounds);
        return c.lo;
    }
    return e;
}
#define PK_CHK_PARAM , const ChkBox &chk
#define PK_CHK_ARG , chk
#define PK_ROW(ptr) Tap<T>::row(chk_row<T>((ptr), chk), dut)
#else
#define PK_CHK_PARAM
#define PK_CHK_ARG
#define PK_ROW(ptr) Tap<T>::row((ptr), dut)
#endif

template <typename T, int NV, int L, uint32_t ROWB, Reuse MODE>
__device__ __forceinline__ void pair_loop(float2 (&acc)[NV][L], const unsigned char *sm, const uint32_t (&cb)[NV],
                                          float sig, float vb, typename Tap<T>::Du dut,
                                          const typename Tap<T>::Wt (&W)[NV] PK_CHK_PARAM)
{
    using R = typename Tap<T>::R;
    R lo[NV], hi[NV];
    float dv;
    uint32_t tv = floor_frac(vb, dv);
#pragma unroll
    for (int n = 0; n < NV; ++n) {
        const unsigned char *e = sm + (cb[n] + tv * ROWB);
        lo[n] = PK_ROW(e);
        hi[n] = PK_ROW(e + ROWB);
    }
#pragma unroll
    for (int n = 0; n < NV; ++n)
        acc[n][0] = Tap<T>::accum(acc[n][0], lo[n], hi[n], make_float2(dv, dv), __float2half2_rn(dv), W[n]);
#pragma unroll
    for (int p = 1; p < L; ++p) {
        const uint32_t tn = floor_frac(fmaf((float)p, sig, vb), dv);
        const uint32_t to = tn * ROWB;
        const float2 dv2 = make_float2(dv, dv);
        const __half2 dvh = __float2half2_rn(dv);
        if constexpr (MODE == Reuse::ANY) {
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                const unsigned char *e = sm + (cb[n] + to);
                lo[n] = PK_ROW(e);
                hi[n] = PK_ROW(e + ROWB);
            }
        } else if constexpr (MODE == Reuse::STEP1) {
            const bool moved = tn != tv;
            tv = tn;
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                const unsigned char *e = sm + (cb[n] + to);
                const R hn = PK_ROW(e + ROWB);
                lo[n] = moved ? hi[n] : lo[n];
                hi[n] = hn;
            }
        } else {
            const uint32_t step = tn - tv;
            tv = tn;
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                const unsigned char *e = sm + (cb[n] + to);
                const R hn = PK_ROW(e + ROWB);
                R ln = step != 0 ? hi[n] : lo[n];
                if (step == 2) ln = PK_ROW(e);
                lo[n] = ln;
                hi[n] = hn;
            }
        }
#pragma unroll
        for (int n = 0; n < NV; ++n) acc[n][p] = Tap<T>::accum(acc[n][p], lo[n], hi[n], dv2, dvh, W[n]);
    }
}

// Writes a z-run: acc[p].x -> voxel k0+p, acc[p].y -> its mirror nz-1-k0-p, of column (i, j)
// of the volume at dst: added (ADD), or stored (a partial volume of a view split).
// GEN (general launches: pair ranges, view split): the output column holds
// nz_out voxels from pair pair0 on; else the whole volume (pair0 = 0, nz_out = nz).
template <int L, bool ADD, bool GEN>
__device__ __forceinline__ void write_run(const PkArgs &a, float *dst, int k0, int i, int j, const float2 *acc)
{
    static_assert(L % 4 == 0, "the vector path stores float4 runs from k0 = a multiple of L");
    const int nz_out = GEN ? a.nz_out : a.nz, pair0 = GEN ? a.pair0 : 0;
    const int pair_end = GEN ? a.pair_end : (a.nz + 1) / 2;
    float *col = dst + ((size_t)i * a.ny + j) * (size_t)nz_out;
    const int lo = k0 - pair0;          // the run's first voxel in the output column
    if ((nz_out & 3) == 0 && (lo & 3) == 0 && k0 + L <= min(a.nz / 2, pair_end)) {
        float4 *pd = reinterpret_cast<float4 *>(col + lo);
        float4 *pm = reinterpret_cast<float4 *>(col + (nz_out - lo - L));
#pragma unroll
        for (int q = 0; q < L / 4; ++q) {
            float4 d = ADD ? pd[q] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            d.x += acc[4 * q].x; d.y += acc[4 * q + 1].x; d.z += acc[4 * q + 2].x; d.w += acc[4 * q + 3].x;
            pd[q] = d;
            float4 m = ADD ? pm[q] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);   // voxels nz-k0-L+4q .. +3: mirror pairs L-1-4q .. L-4-4q
            m.x += acc[L - 1 - 4 * q].y; m.y += acc[L - 2 - 4 * q].y;
            m.z += acc[L - 3 - 4 * q].y; m.w += acc[L - 4 - 4 * q].y;
            pm[q] = m;
        }
    } else {
#pragma unroll
        for (int p = 0; p < L; ++p) {
            const int k = k0 + p;
            if (k < pair_end) {
                const int kd = k - pair0, km = nz_out - 1 - kd;   // voxel k and its mirror nz - 1 - k
                col[kd] = ADD ? col[kd] + acc[p].x : acc[p].x;
                if (a.nz - 1 - k > k) col[km] = ADD ? col[km] + acc[p].y : acc[p].y;
            }
        }
    }
}

// Shared-memory map (offsets from a 128-byte aligned base): full barriers at
// 8 s, empty barriers at 64 + 8 s, the abort flag at 128, the last group
// issued into each stage at 160 + 4 s, stages from 256; a stage is its
// PkGeom (128 bytes reserved) followed by the box.
constexpr uint32_t kPkFull = 0, kPkEmpty = 64, kPkAbort = 128, kPkLast = 160, kPkStage0 = 256, kPkBox = 128;
static_assert(kPkMaxStages * 8 <= 64 && kPkLast + 4 * kPkMaxStages <= kPkStage0, "shared-memory map");

// SPLIT: the general instantiation, for launches that split their view range
// over grid layers (a.part != nullptr) or cover a range of mirror pairs; a
// separate instantiation keeps the whole-volume kernel free of both.
// One block's work: the z-run of L pairs from pair k0 of a 16 x 16 column tile.
template <typename T, int NV, int BW, int L, bool SPLIT>
__device__ __forceinline__ void pk_block(const PkArgs &a, const CUtensorMap &tmap, const int k0)
{
    constexpr uint32_t ES = Tap<T>::ES;
    constexpr int ALIGN = PkT<T>::ALIGN;
    constexpr uint32_t HB = BW * ES;       // one view's part of a box row, bytes
    constexpr uint32_t ROWB = NV * HB;     // box row, bytes
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    const uint32_t sbase = smem_addr(smem_dyn);
    const uint32_t pad = (128u - (sbase & 127u)) & 127u;
    const uint32_t s0 = sbase + pad;                 // shared-window address of the map
    const unsigned char *sm = smem_dyn + pad;        // the same, as a pointer
    const int S = a.stages;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // block coordinates: warp = 16 x 2 patch of columns, 8 warps per 16 x 16 tile.
    // Tiles go in bands of kPkSwizzle tile rows, column by column within a band,
    // so that the blocks resident at one time cover a compact patch of columns
    // (a small detector footprint per view, shared in L2).
    int i0, j0;
    {
        const int t = blockIdx.x, band = t / (kPkSwizzle * a.tiles_x), ty0 = band * kPkSwizzle;
        const int h = min(kPkSwizzle, a.tiles_y - ty0), rem = t - band * kPkSwizzle * a.tiles_x;
        i0 = (rem / h) * kTileX;
        j0 = (ty0 + rem % h) * kTileY;
    }
    const int ci = i0 + (lane & 15), cj = j0 + warp * 2 + (lane >> 4);
    const float ip = (float)ci - a.cx, jp = (float)cj - a.cy, kp0 = (float)k0 - a.cz;

    if (tid == 0) {
        // a bounded wait of this plan ran out (and was not read yet): the
        // results are void, so blocks that start after it do no work
        sts_u32(s0 + kPkAbort, *reinterpret_cast<volatile const unsigned int *>(a.status) & kStatusTimeout);
        prefetch_tmap(&tmap);
        for (int st = 0; st < S; ++st) {
            mbar_init(s0 + kPkFull + 8 * st, 1);
            mbar_init(s0 + kPkEmpty + 8 * st, kThreads / 32);
        }
        fence_barrier_init();
    }
    __syncthreads();
    if (lds_u32_v(s0 + kPkAbort) != 0) return;

    // this block's part of the view range (the whole range without a view split)
    int vbeg = a.view_begin, vcnt = a.view_count;
    if constexpr (SPLIT) {
        vbeg = a.view_begin + (int)(((long long)a.view_count * blockIdx.z) / a.splits);
        vcnt = a.view_begin + (int)(((long long)a.view_count * (blockIdx.z + 1)) / a.splits) - vbeg;
    }
    const int ngroups = NV * vcnt;
    // The block starts its view cycle at view group rot, a fixed function of its
    // place in the launch order: blocks start about a.resident at a time, so a
    // block starting while the others are part-way through the views joins
    // them at the views they are on.  The blocks resident together then read
    // the same views' windows at the same time (in L2) instead of each its
    // own.  The order of the views in a block's sum depends only on the
    // block, so the result is reproducible.
    const long long lin = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    const int rot = vcnt > 0 ? (int)((lin * vcnt / a.resident) % vcnt) : 0;
    // Lane 0 of warp 0: window of group t (own view's footprint of the tile),
    // its terms and the TMA box into stage t % S.
    auto issue = [&](int t) {
        const int st = t % S;
        const uint32_t sg = s0 + kPkStage0 + (uint32_t)st * a.stage_bytes;
        const int qv = t / NV + rot;
        const int s = vbeg + (qv >= vcnt ? qv - vcnt : qv);    // view of the box's slot 0
        const int own = s + (t % NV) * a.pair_view_off;          // the group's own view: slot t mod NV
        const float4 *tp = reinterpret_cast<const float4 *>(a.terms + own);
        const float4 t0 = __ldg(tp), t1 = __ldg(tp + 1);
        float w[4] = {0.0f, 0.0f, 0.0f, 0.0f};                  // FDK weights of the slots' views
#pragma unroll
        for (int n = 0; n < NV; ++n) w[n] = __ldg(&a.terms[s + n * a.pair_view_off].w) * a.wscale;
        // t0 = (A0, A1, A3, B2), t1 = (B3, C0, C1, C3)
        const float ia = (float)i0 - a.cx, ib = ia + (kTileX - 1);
        const float ja = (float)j0 - a.cy, jb = ja + (kTileY - 1);
        float zc[4], uq[4];
        const float cx4[4] = {ia, ib, ia, ib}, cy4[4] = {ja, ja, jb, jb};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            zc[q] = fmaf(t1.y, cx4[q], fmaf(t1.z, cy4[q], t1.w));
            uq[q] = fmaf(t0.x, cx4[q], fmaf(t0.y, cy4[q], t0.z)) / zc[q];
        }
        const float u_lo = fminf(fminf(uq[0], uq[1]), fminf(uq[2], uq[3]));
        const float z_lo = fminf(fminf(zc[0], zc[1]), fminf(zc[2], zc[3]));
        const float z_hi = fmaxf(fmaxf(zc[0], zc[1]), fmaxf(zc[2], zc[3]));
        const float e0 = fmaf(t0.w, kp0, t1.x), e1 = fmaf(t0.w, kp0 + (L - 1), t1.x);
        const float v_lo = fminf(fminf(e0 / z_lo, e0 / z_hi), fminf(e1 / z_lo, e1 / z_hi));
        // box from column u0a (element u0a + 1): TMA needs the element index times
        // its 4 * sizeof(T) bytes on a 16-byte boundary, so u0a + 1 is a multiple of ALIGN
        const int u0a = floor_div((int)floorf(a.uc + u_lo) - kPkMargin + 1, ALIGN) * ALIGN - 1;
        const int v0 = (int)floorf(a.vc + v_lo) - kPkMargin;
        sts_f32x4(sg, t0);
        sts_f32x4(sg + 16, t1);
        sts_f32x4(sg + 32, make_float4(w[0], a.uc - (float)u0a, a.vc - (float)v0, w[1]));
        if constexpr (NV == 4) sts_f32x4(sg + 48, make_float4(w[2], w[3], 0.0f, 0.0f));
        const uint32_t bar = s0 + kPkFull + 8u * st;
        sts_u32(s0 + kPkLast + 4u * st, (uint32_t)t);
        fence_proxy_async_shared();
        mbar_arrive_expect_tx(bar, a.box_tx_bytes);
        const int q = s - a.q_view0;
        if constexpr (NV >= 2)   // the box spans the NV slots (second dimension)
            tma_load_4d(sg + kPkBox, &tmap, 4 * (u0a + 1), 0, v0 - a.row0, q, bar);
        else
            tma_load_3d(sg + kPkBox, &tmap, 4 * (u0a + 1), v0 - a.row0, q, bar);
    };

    // the prologue fills every stage (its lane also records them as the last
    // group issued into each stage, which an aborting warp drains)
    if (warp == 0 && lane == 0)
        for (int t = 0; t < min(S, ngroups); ++t) issue(t);

    float2 acc[NV][L];
#pragma unroll
    for (int n = 0; n < NV; ++n)
#pragma unroll
        for (int p = 0; p < L; ++p) acc[n][p] = make_float2(0.0f, 0.0f);

    // One view group t = NV q + G: wait for its box, form the column terms of
    // the group's own view (the box's slot G) at this thread's column, run the
    // z-run.  Rotational symmetry: the same coordinates belong to the thread's
    // column m in the view of slot (G + m) mod NV, so slot n feeds column
    // (n - G) mod NV.
    bool ok = true;
    auto group = [&](int t, auto g_slot) {
        const int G = g_slot;   // a compile-time constant, or t mod NV
        const int st = t % S;
        const uint32_t parity = (uint32_t)(t / S) & 1u;
        // refill the stage group t - 2 used (every warp finished it by now, or soon)
        const int gn = t - 2 + S;
        if (t >= 2 && gn < ngroups && (t & (kThreads / 32 - 1)) == warp) {
            bool e = true;
            if (lane == 0) {
                e = mbar_wait_lim(s0 + kPkEmpty + 8u * ((t - 2) % S), (uint32_t)((t - 2) / S) & 1u, a.wait_ns);
                if (e) issue(gn);
            }
            ok = __shfl_sync(0xffffffffu, e, 0) != 0;
            if (!ok) return;
        }
        ok = __all_sync(0xffffffffu, t != a.abort_group && mbar_wait_lim(s0 + kPkFull + 8u * st, parity, a.wait_ns));
        if (!ok) return;
        const uint32_t sg = kPkStage0 + (uint32_t)st * a.stage_bytes;
        const float4 *gp = reinterpret_cast<const float4 *>(sm + sg);
        const float4 t0 = gp[0], t1 = gp[1], t2 = gp[2];
        const float4 t3 = NV == 4 ? gp[3] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        // Theorems 2 and 3: z, u and W_dis do not depend on k
        const float z = fmaf(t1.y, ip, fmaf(t1.z, jp, t1.w));
        const float f = rcp_nr(z);
        const float x = fmaf(t0.x, ip, fmaf(t0.y, jp, t0.z));
        float du;
        const uint32_t tu = floor_frac(fmaf(x, f, t2.y), du);
        const float ff = f * f;
        const float wsl[4] = {t2.x, t2.w, t3.x, t3.y};
        typename Tap<T>::Wt Ws[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) Ws[n] = Tap<T>::weight(wsl[n] * ff);
        const float sig = t0.w * f;
        const float vb = fmaf(sig, kp0, fmaf(t1.x, f, t2.z));
        // element (n, cu) at offset base + bits(t_v) * ROWB (mod 2^32): n = bits(t_v) - bias,
        // cu = bits(t_u) - bias
        const uint32_t base = sg + kPkBox + (tu - kFloorBias) * ES - kFloorBias * ROWB;
        // column m takes box slot (m + G) mod NV
        typename Tap<T>::Wt W[NV];
        uint32_t cb[NV];
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            const int n = (m + G) & (NV - 1);
            W[m] = Ws[0];
#pragma unroll
            for (int q = 1; q < NV; ++q)
                if (n == q) W[m] = Ws[q];
            cb[m] = base + (uint32_t)n * HB;
        }
        const typename Tap<T>::Du dut = Tap<T>::frac_u(du);
        // sig < 1 - 2^-10 keeps fp32 rounding of v_{p+1} - v_p below one row; the
        // plan keeps every sig below 1.9 (two rows at most)
        // (FP32 taps keep the reuse across two-row steps; 16-bit taps load both rows,
        // which measured faster for them)
        constexpr Reuse WIDE = sizeof(T) == 4 ? Reuse::STEP2 : Reuse::ANY;
#ifdef IFDK_CHECK
        const ChkBox chk{sm + sg + kPkBox, sm + sg + kPkBox + a.box_tx_bytes, a.status};
#endif
        if (__all_sync(0xffffffffu, sig < 0.9990234375f))
            pair_loop<T, NV, L, ROWB, Reuse::STEP1>(acc, sm, cb, sig, vb, dut, W PK_CHK_ARG);
        else
            pair_loop<T, NV, L, ROWB, WIDE>(acc, sm, cb, sig, vb, dut, W PK_CHK_ARG);
        __syncwarp();
        if (lane == 0) mbar_arrive(s0 + kPkEmpty + 8u * st);
    };
    if constexpr (sizeof(T) == 4) {
        // FP32 taps: one copy of the group body per slot rotation G (constant
        // slot offsets; measured faster for them)
        for (int t = 0; ok && t < ngroups; t += NV) {
            group(t, std::integral_constant<int, 0>{});
            if constexpr (NV >= 2)
                if (ok) group(t + 1, std::integral_constant<int, 1>{});
            if constexpr (NV == 4) {
                if (ok) group(t + 2, std::integral_constant<int, 2>{});
                if (ok) group(t + 3, std::integral_constant<int, 3>{});
            }
        }
    } else {
        // 16-bit taps: one copy for every rotation (the longer z-runs' unrolled
        // body NV times over measured slower: instruction fetch)
        for (int t = 0; ok && t < ngroups; ++t) group(t, t & (NV - 1));
    }
    if (!ok) {
        // record the timeout; every exiting warp waits (bounded) for the last box
        // issued into each stage, so the last warp to leave the block leaves no
        // copy in flight (a warp issues nothing after it left)
        if (lane == 0) {
            atomicOr(a.status, kStatusTimeout);
            for (int st = 0; st < min(S, ngroups); ++st) {
                const int t = (int)lds_u32_v(s0 + kPkLast + 4u * st);
                mbar_wait_lim(s0 + kPkFull + 8u * st, (uint32_t)(t / S) & 1u, kPkDrainNs);
            }
        }
        return;
    }
    if (a.wunscale != 1.0f) {
#pragma unroll
        for (int n = 0; n < NV; ++n)
#pragma unroll
            for (int p = 0; p < L; ++p) acc[n][p] = make_float2(acc[n][p].x * a.wunscale, acc[n][p].y * a.wunscale);
    }
    if (ci < a.nx_cols && cj < a.ny_cols) {
        // the thread's columns: (ci, cj) and its images under the scan's turn by
        // 2 pi / NV (a quarter turn maps (i, j) to (nx-1-j, i); nx = ny for NV = 4)
        int cx[NV], cy[NV];
        cx[0] = ci;
        cy[0] = cj;
        if constexpr (NV == 2) {
            cx[1] = a.nx - 1 - ci;
            cy[1] = a.ny - 1 - cj;
        }
        if constexpr (NV == 4) {
            cx[1] = a.nx - 1 - cj; cy[1] = ci;
            cx[2] = a.nx - 1 - ci; cy[2] = a.ny - 1 - cj;
            cx[3] = cj;            cy[3] = a.ny - 1 - ci;
        }
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            if constexpr (!SPLIT) {
                write_run<L, true, false>(a, a.vol, k0, cx[m], cy[m], acc[m]);
            } else if (a.part != nullptr) {
                write_run<L, false, true>(a, a.part + blockIdx.z * a.part_stride, k0, cx[m], cy[m], acc[m]);
            } else {
                write_run<L, true, true>(a, a.vol, k0, cx[m], cy[m], acc[m]);
            }
        }
    }
}

// z-blocks 0 .. zfull - 1 take L pairs each; the blocks after them take the
// remaining npairs - zfull L pairs kPkTailL at a time, so that no block runs
// pairs past the volume's middle.
template <typename T, int NV, int BW, int L, bool SPLIT>
__global__ void __launch_bounds__(kThreads, pk_blocks(NV))
    bp_packed_kernel(const PkArgs a, const __grid_constant__ CUtensorMap tmap)
{
    const int pair0 = SPLIT ? a.pair0 : 0;
    if constexpr (L == kPkTailL) {
        pk_block<T, NV, BW, L, SPLIT>(a, tmap, pair0 + (int)blockIdx.y * L);
    } else {
        if ((int)blockIdx.y < a.zfull)
            pk_block<T, NV, BW, L, SPLIT>(a, tmap, pair0 + (int)blockIdx.y * L);
        else
            pk_block<T, NV, BW, kPkTailL, SPLIT>(a, tmap, pair0 + a.zfull * L + ((int)blockIdx.y - a.zfull) * kPkTailL);
    }
}

// Packing: element e of row r of view s, column c = e - 1:
// (Q[r][c], Q[2vc-r][c], Q[r][c+1] - Q[r][c], Q[2vc-r][c+1] - Q[2vc-r][c]),
// the differences formed in FP32 and rounded once to T; for BF16
// (Q[r][c], Q[2vc-r][c], Q[r][c+1], Q[2vc-r][c+1]), the stored values.
__device__ __forceinline__ uint32_t bits16(__half x) { return __half_as_ushort(x); }
__device__ __forceinline__ uint32_t bits16(__nv_bfloat16 x) { return __bfloat16_as_ushort(x); }
struct PackArgs {
    long long n_elems;   // n_views * rows * nu_p
    int nv, nu, nu_p, rows, row0, two_vc;
};

template <typename T>
__global__ void __launch_bounds__(256) pack_kernel(const T *__restrict__ Q, T *__restrict__ P, const PackArgs a)
{
    for (long long e = blockIdx.x * 256ll + threadIdx.x; e < a.n_elems; e += (long long)gridDim.x * 256) {
        const int c = (int)(e % a.nu_p) - 1;
        const long long sr = e / a.nu_p;
        const int r = (int)(sr % a.rows) + a.row0;
        const long long s = sr / a.rows;
        const T *qv = Q + s * a.nv * (long long)a.nu;
        const int rm = a.two_vc - r;
        const bool dr = r >= 0 && r < a.nv, mr = rm >= 0 && rm < a.nv;
        const bool c0 = c >= 0 && c < a.nu, c1 = c + 1 < a.nu;   // c + 1 >= 0 always
        const float q0 = dr && c0 ? Storage<T>::to_float(qv[(long long)r * a.nu + c]) : 0.0f;
        const float q1 = mr && c0 ? Storage<T>::to_float(qv[(long long)rm * a.nu + c]) : 0.0f;
        const float q2 = dr && c1 ? Storage<T>::to_float(qv[(long long)r * a.nu + c + 1]) : 0.0f;
        const float q3 = mr && c1 ? Storage<T>::to_float(qv[(long long)rm * a.nu + c + 1]) : 0.0f;
        const T v0 = Storage<T>::from_float(q0), v1 = Storage<T>::from_float(q1);
        constexpr bool kRawTaps = std::is_same<T, __nv_bfloat16>::value;
        const T v2 = Storage<T>::from_float(kRawTaps ? q2 : q2 - q0);
        const T v3 = Storage<T>::from_float(kRawTaps ? q3 : q3 - q1);
        T *d = P + e * 4;
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(d) = make_float4(v0, v1, v2, v3);
        } else {
            *reinterpret_cast<uint2 *>(d) = make_uint2(bits16(v0) | (bits16(v1) << 16), bits16(v2) | (bits16(v3) << 16));
        }
    }
}

// View split: vol += part[0] + part[1] + ... + part[S-1], element by element in
// part order (the same order every call, so the result is reproducible).
__global__ void __launch_bounds__(256) split_reduce_kernel(float *vol, const float *part, size_t n, size_t stride,
                                                           int S)
{
    const size_t step = (size_t)gridDim.x * blockDim.x, n4 = n / 4;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (size_t i = t0; i < n4; i += step) {
        float4 v = reinterpret_cast<float4 *>(vol)[i];
        for (int c = 0; c < S; ++c) {
            const float4 q = __ldcs(reinterpret_cast<const float4 *>(part + c * stride) + i);
            v.x += q.x; v.y += q.y; v.z += q.z; v.w += q.w;
        }
        reinterpret_cast<float4 *>(vol)[i] = v;
    }
    for (size_t i = 4 * n4 + t0; i < n; i += step) {
        float v = vol[i];
        for (int c = 0; c < S; ++c) v += part[c * stride + i];
        vol[i] = v;
    }
}

// Parts of the view range per launch: enough to fill one wave of the GPU when
// the grid alone covers at most half of it, each part at least kPkSplitMinUnits
// pairs (or views), at most the partial volumes the plan holds.
int pk_splits(const ifdk_plan_s *p, const PkLaunch &b, int units, int grid_y)
{
    if (!p->d_split || p->view_split_max == 1) return 1;
    const long long blocks = (long long)b.grid_x * grid_y, want = (long long)p->n_sm * pk_blocks(b.nv);
    if (blocks * 2 > want) return 1;
    long long S = std::min<long long>((want + blocks - 1) / blocks, p->split_cap);
    if (p->view_split_max >= 2) S = std::min<long long>(S, p->view_split_max);
    S = std::min<long long>(S, units / kPkSplitMinUnits);
    return S >= 2 ? (int)S : 1;
}

// Host sizing of the packed kernel: windows from analytic FP64 bounds of the
// largest detector footprint of any block over any view.
PkLaunch size_packed(const ifdk_plan_s *p, int q_dtype, int nv)
{
    const ifdk_geometry &g = p->g;
    PkLaunch b{};
    b.path = 0;
    b.nv = nv;
    const int es = (int)dtype_size(q_dtype);
    b.align = q_dtype == IFDK_F32 ? 1 : 2;
    const int ny_cols = nv >= 2 ? g.ny / 2 : g.ny, nx_cols = nv == 4 ? g.nx / 2 : g.nx;
    const int tiles_x = (nx_cols + kTileX - 1) / kTileX, tiles_y = (ny_cols + kTileY - 1) / kTileY;
    const int L = pk_pairs(nv, q_dtype), npairs = (g.nz + 1) / 2;
    b.grid_x = tiles_x * tiles_y;
    b.grid_y = pk_zblocks(npairs, L);
    if (!p->fold_ok) return b;
    if (nv == 2 && (!p->half_turn || g.ny % 2 != 0)) return b;
    // a quarter turn maps the column grid onto itself: square grid, equal pitches, even size;
    // quads are built for FP16 storage only (four columns' FP32 runs and four views' wider
    // taps do not fit the registers of FP32 / BF16 taps without spilling)
    if (nv == 4 && (!p->quarter_turn || g.nx != g.ny || g.nx % 2 != 0 || g.dx != g.dy || q_dtype != IFDK_F16))
        return b;
    const double cx = (g.nx - 1) / 2.0, cy = (g.ny - 1) / 2.0, cz = (g.nz - 1) / 2.0;
    const double xa = cx * g.dx, xb = (tiles_x * kTileX - 1 - cx) * g.dx;
    const double ya = cy * g.dy, yb = (tiles_y * kTileY - 1 - cy) * g.dy;
    const double rxy = std::sqrt(std::max(xa * xa, xb * xb) + std::max(ya * ya, yb * yb));
    const double cmin = g.sid - rxy;
    if (cmin < 0.1 * g.sid) return b;
    const double et = std::hypot((kTileX - 1) * g.dx, (kTileY - 1) * g.dy);
    const double wu = g.sdd / g.du * et * (1.0 / cmin + 2.0 * rxy / (cmin * cmin));
    // a block may start at any pair (pair-range launches) and run L pairs on
    const double kmax = std::max(cz, (double)(npairs + L - 2) - cz);
    const double b2 = g.sdd * g.dz / g.dv;
    if (b2 / cmin >= 1.9) return b;   // rows per voxel step (the largest sig) below 2
    const double hv = b2 * (L - 1) / cmin + b2 * kmax * et / (cmin * cmin);
    b.fold_w = (int)std::ceil(wu) + 2 * kPkMargin + 2;
    b.box_h = (int)std::ceil(hv) + 2 * kPkMargin + 3;
    const int need = b.fold_w + b.align - 1;   // the window starts up to align - 1 into the box
    b.bw = need <= kPkBoxS ? kPkBoxS : kPkBoxL;
    if (need > kPkBoxL || b.box_h > 256) return b;
    const size_t box = (size_t)b.box_h * nv * b.bw * 4 * es;
    b.stage_bytes = (kPkBox + box + 127) / 128 * 128;
    // as many stages as keep pk_blocks(nv) blocks per SM (228 KiB of shared
    // memory per SM, 1 KiB of it reserved per block), at most kPkMaxStages
    const size_t budget = 228 * 1024 / pk_blocks(nv) - 1024;
    b.stages = (int)std::min<size_t>(kPkMaxStages, (budget - 128 - kPkStage0) / b.stage_bytes);
    if (b.stages < 3) b.stages = 3;   // fewer blocks per SM rather than a shallower ring
    b.smem = 128 + kPkStage0 + (size_t)b.stages * b.stage_bytes;
    if (b.smem > 220 * 1024) return b;
    if ((size_t)g.np * p->pk_rows * p->pk_nu * 4 * es >= ((size_t)1 << 40) || b.grid_y > 65535) return b;
    b.pairs = L;
    b.path = 1;
    return b;
}

template <typename T, int NV, int BW>
int launch_packed_t(ifdk_plan_s *p, const PkLaunch &b, const void *Qp, int s_begin, int s_count, int q_view0,
                    int q_pair_off, int q_views, float *vol, cudaStream_t stream, const PkZRange &zr)
{
    const ifdk_geometry &g = p->g;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return IFDK_ERR_CUDA;
    const cuuint64_t es = sizeof(T);
    const cuuint64_t row_bytes = (cuuint64_t)p->pk_nu * 4 * es, view_bytes = row_bytes * p->pk_rows;
    CUtensorMap tmap;
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r;
    if (NV >= 2) {
        // x (elements), slot (view s -> s + np/NV -> ...), row, view
        const cuuint64_t dims[4] = {(cuuint64_t)p->pk_nu * 4, (cuuint64_t)NV, (cuuint64_t)p->pk_rows,
                                    (cuuint64_t)q_views};
        const cuuint64_t strides[3] = {(cuuint64_t)q_pair_off * view_bytes, row_bytes, view_bytes};
        const cuuint32_t box[4] = {(cuuint32_t)(4 * BW), (cuuint32_t)NV, (cuuint32_t)b.box_h, 1};
        r = enc(&tmap, PkT<T>::TMA, 4, const_cast<void *>(Qp), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        const cuuint64_t dims[3] = {(cuuint64_t)p->pk_nu * 4, (cuuint64_t)p->pk_rows, (cuuint64_t)q_views};
        const cuuint64_t strides[2] = {row_bytes, view_bytes};
        const cuuint32_t box[3] = {(cuuint32_t)(4 * BW), (cuuint32_t)b.box_h, 1};
        r = enc(&tmap, PkT<T>::TMA, 3, const_cast<void *>(Qp), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return IFDK_ERR_CUDA;
    PkArgs a;
    a.vol = vol;
    a.terms = p->d_terms;
    a.status = p->d_status;
    a.wait_ns = p->wait_ns;
    a.abort_group = p->test_abort_group;
    a.resident = p->n_sm * pk_blocks(NV);
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
    a.ny_cols = NV >= 2 ? g.ny / 2 : g.ny;
    a.nx_cols = NV == 4 ? g.nx / 2 : g.nx;
    a.tiles_x = (a.nx_cols + kTileX - 1) / kTileX;
    a.tiles_y = (a.ny_cols + kTileY - 1) / kTileY;
    a.view_begin = s_begin;
    a.view_count = s_count;
    a.q_view0 = q_view0;
    a.q_pair_off = q_pair_off;
    a.pair_view_off = g.np / NV;
    a.box_h = b.box_h;
    a.stages = b.stages;
    a.row0 = p->pk_row0;
    a.cx = (float)((g.nx - 1) / 2.0); a.cy = (float)((g.ny - 1) / 2.0); a.cz = (float)((g.nz - 1) / 2.0);
    a.uc = (float)p->uc; a.vc = (float)p->vc;
    a.wscale = sizeof(T) == 2 && PkT<T>::TMA == CU_TENSOR_MAP_DATA_TYPE_FLOAT16 ? p->pk_wscale : 1.0f;
    a.wunscale = 1.0f / a.wscale;
    a.stage_bytes = (uint32_t)b.stage_bytes;
    a.box_tx_bytes = (uint32_t)((size_t)b.box_h * NV * BW * 4 * es);
    constexpr int L = pk_pairs(NV, PkT<T>::CODE);
    const int npairs = (g.nz + 1) / 2, pcount = zr.pcount < 0 ? npairs : zr.pcount;
    a.pair0 = zr.pcount < 0 ? 0 : zr.pair0;
    a.pair_end = a.pair0 + pcount;
    a.nz_out = zr.pcount < 0 ? g.nz : zr.nz_out;
    a.zfull = pcount / L;
    const int grid_y = pk_zblocks(pcount, L);
    if (grid_y == 0) return IFDK_OK;
    const int S = pk_splits(p, b, s_count, grid_y);
    a.part = S > 1 ? p->d_split : nullptr;
    a.part_stride = p->split_stride;
    a.splits = S;
    const bool general = S > 1 || zr.pcount >= 0;
    void (*kern)(const PkArgs, const CUtensorMap) =
        general ? bp_packed_kernel<T, NV, BW, L, true> : bp_packed_kernel<T, NV, BW, L, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.smem) != cudaSuccess)
        return IFDK_ERR_CUDA;
    kern<<<dim3(b.grid_x, grid_y, S), kThreads, b.smem, stream>>>(a, tmap);
    if (cudaGetLastError() != cudaSuccess) return IFDK_ERR_CUDA;
    if (S > 1) {
        const size_t n = (size_t)g.nx * g.ny * a.nz_out;
        const size_t blocks = std::min<size_t>((n / 4 + 255) / 256 + 1, (size_t)p->n_sm * 8);
        split_reduce_kernel<<<(unsigned)blocks, 256, 0, stream>>>(vol, p->d_split, n, p->split_stride, S);
        if (cudaGetLastError() != cudaSuccess) return IFDK_ERR_CUDA;
    }
    return IFDK_OK;
}

template <typename T, int NV>
int launch_packed_bw(ifdk_plan_s *p, const PkLaunch &b, const void *Qp, int s_begin, int s_count, int q_view0,
                     int q_pair_off, int q_views, float *vol, cudaStream_t stream, const PkZRange &zr)
{
    return b.bw == kPkBoxS ? launch_packed_t<T, NV, kPkBoxS>(p, b, Qp, s_begin, s_count, q_view0, q_pair_off, q_views,
                                                             vol, stream, zr)
                           : launch_packed_t<T, NV, kPkBoxL>(p, b, Qp, s_begin, s_count, q_view0, q_pair_off, q_views,
                                                             vol, stream, zr);
}

template <int NV>
int launch_packed(ifdk_plan_s *p, const void *Qp, int q_dtype, int s_begin, int s_count, int q_view0, int q_pair_off,
                  int q_views, float *vol, cudaStream_t stream, const PkZRange &zr)
{
    if (s_count <= 0) return IFDK_OK;
    const PkLaunch &b = NV == 4 ? p->pk4[q_dtype] : (NV == 2 ? p->pk2[q_dtype] : p->pk[q_dtype]);
    if (!b.path) return IFDK_ERR_UNSUPPORTED;
    if constexpr (NV == 4) {   // quads: FP16 storage only (size_packed)
        if (q_dtype != IFDK_F16) return IFDK_ERR_UNSUPPORTED;
        return launch_packed_bw<__half, NV>(p, b, Qp, s_begin, s_count, q_view0, q_pair_off, q_views, vol, stream, zr);
    } else {
        switch (q_dtype) {
        case IFDK_F32:
            return launch_packed_bw<float, NV>(p, b, Qp, s_begin, s_count, q_view0, q_pair_off, q_views, vol, stream,
                                               zr);
        case IFDK_F16:
            return launch_packed_bw<__half, NV>(p, b, Qp, s_begin, s_count, q_view0, q_pair_off, q_views, vol, stream,
                                                zr);
        default:
            return launch_packed_bw<__nv_bfloat16, NV>(p, b, Qp, s_begin, s_count, q_view0, q_pair_off, q_views, vol,
                                                       stream, zr);
        }
    }
}

}  // namespace

int plan_view_split(ifdk_plan_s *p)
{
    const ifdk_geometry &g = p->g;
    if (cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
        return IFDK_ERR_CUDA;
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    p->split_stride = (nvox + 3) / 4 * 4;   // keeps every partial volume 16-byte aligned
    bool small = false;
    for (int d = 0; d < 3; ++d)
        for (const PkLaunch *b : {&p->pk[d], &p->pk2[d], &p->pk4[d]})
            if (b->path && (long long)b->grid_x * b->grid_y * 2 <= (long long)p->n_sm * pk_blocks(b->nv)) small = true;
    if (!small) return IFDK_OK;
    const size_t cap = std::min<size_t>(kPkMaxSplits, kPkSplitBytes / (p->split_stride * sizeof(float)));
    if (cap < 2) return IFDK_OK;
    if (cudaMalloc(&p->d_split, cap * p->split_stride * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return IFDK_ERR_NOMEM;
    }
    p->split_cap = (int)cap;
    return IFDK_OK;
}

int packed_view_split(const ifdk_plan_s *p, int q_dtype, int units, int nv)
{
    const PkLaunch &b = nv == 4 ? p->pk4[q_dtype] : (nv == 2 ? p->pk2[q_dtype] : p->pk[q_dtype]);
    return b.path ? pk_splits(p, b, units, b.grid_y) : 1;
}

void split_half_turn(int np, int b, int e, int *m)
{
    const int h = np / 2;
    *m = b;
    if (np < 2 || np % 2 != 0 || b >= h) return;
    const int mm = std::min(h, e - h);
    if (mm > b) *m = mm;
}

void plan_packed(ifdk_plan_s *p)
{
    // rows r0 = min(0, 2 vc - (nv - 1)) .. floor(vc) + 2: every row a voxel
    // k <= nz / 2 taps (v <= vc, plus FP32 rounding), and rows above the
    // detector whose mirror lies on it
    p->pk_row0 = std::min(0, p->two_vc - (p->g.nv - 1));
    p->pk_rows = p->fold_ok ? (int)std::floor(p->vc) + 3 - p->pk_row0 : 0;
    p->pk_nu = (p->g.nu + 2) / 2 * 2;   // columns -1 .. nu - 1, rounded up to even
    // FP16 weights: W = w_s f^2 <= max w_s / z_min^2 with z_min >= d - r_xy (r_xy the
    // largest voxel distance from the axis); scale by 2^k so that it lies in [1, 2)
    {
        const ifdk_geometry &g = p->g;
        const double hx = 0.5 * (g.nx - 1) * g.dx, hy = 0.5 * (g.ny - 1) * g.dy;
        const double zmin = g.sid - std::sqrt(hx * hx + hy * hy);
        double wmax = 0.0;
        for (const ViewTerms &t : p->terms) wmax = std::max(wmax, (double)std::fabs(t.w));
        const double Wmax = wmax / (zmin * zmin);
        p->pk_wscale = Wmax > 0.0 ? (float)std::ldexp(1.0, -(int)std::floor(std::log2(Wmax))) : 1.0f;
    }
    for (int t = 0; t < 3; ++t) {
        p->pk[t] = size_packed(p, t, 1);
        p->pk2[t] = p->pk[t].path ? size_packed(p, t, 2) : PkLaunch{};
        p->pk4[t] = p->pk2[t].path ? size_packed(p, t, 4) : PkLaunch{};
    }
}

size_t packed_view_bytes(const ifdk_plan_s *p, int q_dtype)
{
    return (size_t)p->pk_rows * p->pk_nu * 4 * dtype_size(q_dtype);
}

int launch_pack(ifdk_plan_s *p, const void *Q, int q_dtype, int n_views, void *Qp, cudaStream_t stream)
{
    if (n_views <= 0) return IFDK_OK;
    PackArgs a;
    a.nv = p->g.nv; a.nu = p->g.nu; a.nu_p = p->pk_nu; a.rows = p->pk_rows; a.row0 = p->pk_row0;
    a.two_vc = p->two_vc;
    a.n_elems = (long long)n_views * a.rows * a.nu_p;
    const long long blocks = std::min<long long>((a.n_elems + 255) / 256, 152ll * 64);
    switch (q_dtype) {
    case IFDK_F32:
        pack_kernel<float><<<(unsigned)blocks, 256, 0, stream>>>(static_cast<const float *>(Q), static_cast<float *>(Qp), a);
        break;
    case IFDK_F16:
        pack_kernel<__half><<<(unsigned)blocks, 256, 0, stream>>>(static_cast<const __half *>(Q), static_cast<__half *>(Qp), a);
        break;
    default:
        pack_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, stream>>>(static_cast<const __nv_bfloat16 *>(Q),
                                                                       static_cast<__nv_bfloat16 *>(Qp), a);
    }
    return cudaGetLastError() == cudaSuccess ? IFDK_OK : IFDK_ERR_CUDA;
}

int launch_packed_pairs(ifdk_plan_s *p, const void *Qp, int q_dtype, int s_begin, int s_count, int q_view0,
                        int q_pair_off, int q_views, float *vol, cudaStream_t stream)
{
    return launch_packed<2>(p, Qp, q_dtype, s_begin, s_count, q_view0, q_pair_off, q_views, vol, stream, PkZRange{});
}

int launch_packed_quads(ifdk_plan_s *p, const void *Qp, int q_dtype, int s_begin, int s_count, int q_view0,
                        int q_slot_off, int q_views, float *vol, cudaStream_t stream)
{
    return launch_packed<4>(p, Qp, q_dtype, s_begin, s_count, q_view0, q_slot_off, q_views, vol, stream, PkZRange{});
}

int launch_backproject_packed(ifdk_plan_s *p, const void *Qp, int q_dtype, int view_begin, int view_count,
                              int q_view0, int q_views, float *vol, cudaStream_t stream, const PkZRange &zr)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    const int b = view_begin, e = view_begin + view_count, h = p->g.np / 2;
    // the whole scan in quarter-turn quads (s, s + np/4, s + np/2, s + 3np/4), s < np/4
    if (p->use_quarter_turn && p->pk4[q_dtype].path && b == 0 && e == p->g.np && q_view0 == 0 &&
        q_views == p->g.np)
        return launch_packed<4>(p, Qp, q_dtype, 0, p->g.np / 4, 0, p->g.np / 4, p->g.np, vol, stream, zr);
    int m = b;
    if (p->use_half_turn && p->pk2[q_dtype].path) split_half_turn(p->g.np, b, e, &m);
    if (m == b) return launch_packed<1>(p, Qp, q_dtype, b, view_count, q_view0, 0, q_views, vol, stream, zr);
    // views s in [b, m) with their partners s + h; then the unpaired [m, b + h) and [m + h, e)
    int rc = launch_packed<2>(p, Qp, q_dtype, b, m - b, q_view0, h, q_views, vol, stream, zr);
    if (rc == IFDK_OK) rc = launch_packed<1>(p, Qp, q_dtype, m, b + h - m, q_view0, 0, q_views, vol, stream, zr);
    if (rc == IFDK_OK) rc = launch_packed<1>(p, Qp, q_dtype, m + h, e - m - h, q_view0, 0, q_views, vol, stream, zr);
    return rc;
}

}  // namespace ifdk
