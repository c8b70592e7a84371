// Filtering stage (Algorithm 1 of the iFDK paper) on the 5th-generation
// tensor cores, as a dense Toeplitz GEMM over detector rows.
//
// Summation by parts: with the weighted row w = F_cos E (w = 0 outside
// [0, nu)), its first difference d(k) = w(k) - w(k-1) for k in [0, nu], and
// the running sum of the Ram-Lak taps g(m) = sum_{j <= m} h(j)
// (j from -(nu-1)), the exact linear convolution of Algorithm 1 is
//     Q(u) = sum_k h(u - k) w(k) = sum_{k=0}^{nu} g(u - k) d(k).
// The ramp filter removes the large smooth part of each row: at 2048 pixels
// |w| is ~1400 x |Q|, so in the first form every rounding of w or of a
// partial sum is amplified ~1400 times; d is ~6 x |Q| and g is bounded by
// 1/8 (it decays like 1/(2 pi^2 m)), so the second form is well conditioned
// and FP32 accumulation suffices.  The GEMM is Q = D . G with K = nu + 1.
//
// Both operands are split into BF16 terms (each the rounded remainder of the
// previous) and the products of data term i and tap term j are accumulated in
// FP32 in tensor memory: s = 1: (0,0); s = 2: i + j <= 1; s = 3: i + j <= 2
// (FP32 d is exactly three BF16 terms, the taps get 24 bits).  d is formed
// from w as a double-float (FMA two-product of E with the hi/lo F_cos table),
// so that FP32 rounding of w is not differenced.
//
// Kernels: a pre-pass writes d of a chunk of rows as s BF16 planes into a
// caller-provided workspace; the GEMM kernel computes one 128 x 128 output
// tile per block: one lane streams, per K block of 64, all s data planes and
// all s tap planes by TMA (128-byte swizzle) into one stage of an mbarrier
// ring, so every plane is read once per K block whatever the number of term
// products; one lane issues tcgen05.mma (M = 128, N = 128, K = 16) for every
// term pair of the stage into four TMEM accumulators (see acc_of), and the
// four warps read them back (tcgen05.ld), add them and store the storage
// type.
#include <cstring>

#include "ifdk_device.cuh"
#include "ifdk_internal.h"

namespace ifdk {
namespace {

constexpr int kTcM = 128, kTcN = 128, kTcK = 64;
constexpr int kTcThreads = 128;
constexpr uint32_t kTileA = kTcM * kTcK * 2, kTileB = kTcN * kTcK * 2;   // 16 KiB each (one plane)
constexpr int kTcMaxStages = 6;
// stages of s data planes + s tap planes (32 KiB per plane pair) within 192 KiB
constexpr int tc_stages(int planes) { return planes == 3 ? 2 : (planes == 2 ? 3 : 6); }
constexpr uint32_t tc_stage_bytes(int planes) { return (uint32_t)planes * (kTileA + kTileB); }
constexpr size_t tc_smem(int planes) { return 1024 + (size_t)tc_stages(planes) * tc_stage_bytes(planes) + 256; }
constexpr int kAccs = 4;
constexpr uint32_t kTmemCols = kAccs * kTcN;   // four FP32 accumulators of kTcN columns

// TMEM accumulator of unit (K block kb, term pair q): the leading product
// (q = 0) rotates over three accumulators by K block, the small cross
// products share the fourth.  The tensor cores' accumulation into TMEM is
// not round-to-nearest FP32, and its error grows with the number of MMAs
// accumulated at a given magnitude; splitting the steps this way and adding
// the four in FP32 in the epilogue keeps it ~20x below one accumulator's.
__device__ __forceinline__ int acc_of(int kb, int q) { return q == 0 ? kb % 3 : 3; }

struct TcArgs {
    void *Q;
    unsigned int *status;
    unsigned long long wait_ns;
    long long row0;       // first output row of this chunk
    int nrows;            // rows in this chunk
    int nu, nk, npairs;   // K blocks of 64, term pairs
    int planes, stages;   // split terms (planes of each operand per stage), ring depth
    unsigned int *view_max;   // [np] bits of max |Q| per view (nullptr: not taken)
    int nv;
};

// Term pairs (data i, tap j): s = 1, 2, 3 use the first 1, 3, 6.
__device__ __forceinline__ void term_pair(int q, int &i, int &j)
{
    i = (q == 2 || q == 4) ? 1 : (q == 5 ? 2 : 0);
    j = (q == 1 || q == 4) ? 1 : (q == 3 ? 2 : 0);
}

template <typename TQ> __device__ __forceinline__ void store_row32(TQ *dst, const uint32_t (&r)[32], int n);
template <> __device__ __forceinline__ void store_row32<float>(float *dst, const uint32_t (&r)[32], int n)
{
    if (n == 32 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            reinterpret_cast<uint4 *>(dst)[q] = make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < 32; ++q)   // unrolled: r stays in registers
            if (q < n) dst[q] = __uint_as_float(r[q]);
    }
}
template <typename T16>
__device__ __forceinline__ void store_row32_16(T16 *dst, const uint32_t (&r)[32], int n)
{
    if (n == 32 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const T16 lo = Storage<T16>::from_float(__uint_as_float(r[8 * q + 2 * e]));
                const T16 hi = Storage<T16>::from_float(__uint_as_float(r[8 * q + 2 * e + 1]));
                w[e] = (uint32_t)(*reinterpret_cast<const uint16_t *>(&lo)) |
                       ((uint32_t)(*reinterpret_cast<const uint16_t *>(&hi)) << 16);
            }
            reinterpret_cast<uint4 *>(dst)[q] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 32; ++q)
            if (q < n) dst[q] = Storage<T16>::from_float(__uint_as_float(r[q]));
    }
}
template <> __device__ __forceinline__ void store_row32<__half>(__half *dst, const uint32_t (&r)[32], int n)
{
    store_row32_16(dst, r, n);
}
template <> __device__ __forceinline__ void store_row32<__nv_bfloat16>(__nv_bfloat16 *dst, const uint32_t (&r)[32],
                                                                      int n)
{
    store_row32_16(dst, r, n);
}

template <typename TQ>
__global__ void __launch_bounds__(kTcThreads, 1)
    filter_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    const uint32_t sbase = smem_addr(smem_dyn);
    const uint32_t s0 = sbase + ((1024u - (sbase & 1023u)) & 1023u);   // 128-byte swizzle wants 1 KiB alignment
    const int S = a.stages;
    const uint32_t stage_bytes = (uint32_t)a.planes * (kTileA + kTileB);
    // stage s: data planes at s0 + s * stage_bytes, then the tap planes
    const uint32_t full = s0 + (uint32_t)S * stage_bytes, empty = full + 8 * kTcMaxStages,
                   accum = empty + 8 * kTcMaxStages;
    const uint32_t tslot = accum + 8, abort_flag = tslot + 4;   // abort_flag + 4: accumulators written
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // column tiles fastest: the npad / 128 blocks of one row tile run side by side
    // and share its data planes in L2 (read from DRAM once, not once per column tile)
    const int n_tile = blockIdx.x, m_tile = blockIdx.y;
    const int units = a.nk;   // one unit = one K block, all planes of both operands

    if (tid == 0) {
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
        for (int s = 0; s < S; ++s) {
            mbar_init(full + 8 * s, 1);
            mbar_init(empty + 8 * s, 1);
        }
        mbar_init(accum, 1);
        asm volatile("st.shared.u32 [%0], %1;" ::"r"(abort_flag), "r"(0u) : "memory");
        fence_barrier_init();
    }
    if (warp == 0) tc::alloc(tslot, kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    uint32_t tmem;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(tmem) : "r"(tslot) : "memory");

    if (warp == 0 && lane == 0) {
        // TMA producer: K block u (every data plane, every tap plane) into stage u % S
        for (int u = 0; u < units; ++u) {
            const int s = u % S;
            if (!mbar_wait_bounded(empty + 8 * s, ((u / S) & 1) ^ 1, a.wait_ns)) {
                asm volatile("st.shared.u32 [%0], %1;" ::"r"(abort_flag), "r"(1u) : "memory");
                break;
            }
            const uint32_t st = s0 + (uint32_t)s * stage_bytes;
            mbar_arrive_expect_tx(full + 8 * s, stage_bytes);
            tma_load_3d(st, &tmA, u * kTcK, m_tile * kTcM, 0, full + 8 * s);
            tma_load_3d(st + (uint32_t)a.planes * kTileA, &tmB, u * kTcK, n_tile * kTcN, 0, full + 8 * s);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: per term pair (i, j) of a K block, 4 x (M128 N128 K16) of data
        // plane i and tap plane j into TMEM accumulator acc_of(kb, q)
        constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcM, kTcN);
        uint32_t started = 0;   // bit c: accumulator c has been written
        for (int u = 0; u < units; ++u) {
            const int s = u % S;
            if (!mbar_wait_bounded(full + 8 * s, (u / S) & 1, a.wait_ns)) {
                asm volatile("st.shared.u32 [%0], %1;" ::"r"(abort_flag), "r"(1u) : "memory");
                break;
            }
            tc::fence_after();
            const uint32_t st = s0 + (uint32_t)s * stage_bytes;
            for (int q = 0; q < a.npairs; ++q) {
                int ti, tj;
                term_pair(q, ti, tj);
                const int c = acc_of(u, q);
                const uint32_t d = tmem + (uint32_t)c * kTcN;
                const uint64_t da = tc::desc_sw128(st + (uint32_t)ti * kTileA);
                const uint64_t db = tc::desc_sw128(st + (uint32_t)a.planes * kTileA + (uint32_t)tj * kTileB);
#pragma unroll
                for (int kk = 0; kk < kTcK / 16; ++kk) {   // +32 bytes along K = +2 in the address field
                    tc::mma_f16(d, da + 2 * kk, db + 2 * kk, idesc, (started >> c) & 1u);
                    started |= 1u << c;
                }
            }
            tc::commit(empty + 8 * s);
        }
        asm volatile("st.shared.u32 [%0], %1;" ::"r"(abort_flag + 4), "r"(started) : "memory");
        tc::commit(accum);   // arrives when every MMA issued above has completed
    }
    __syncwarp();

    // epilogue: warp w reads TMEM lanes 32w..32w+31 (tile rows), 32 columns at a time
    const bool ok = mbar_wait_bounded(accum, 0, a.wait_ns);
    tc::fence_after();
    uint32_t aborted;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(aborted) : "r"(abort_flag) : "memory");
    uint32_t started;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(started) : "r"(abort_flag + 4) : "memory");
    const int lrow = m_tile * kTcM + warp * 32 + lane;
    const long long grow = a.row0 + lrow;
    TQ *Q = static_cast<TQ *>(a.Q);
    const bool row_ok = ok && !aborted && lrow < a.nrows;
    uint32_t amax = 0u;   // bits of max |Q| over this thread's row of the tile (FP32, before the cast)
#pragma unroll 1
    for (int cb = 0; cb < kTcN / 32; ++cb) {
        // sum of the accumulators written, in FP32 (round to nearest)
        uint32_t r[32], t[32];
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32);
#pragma unroll
        for (int q = 0; q < 32; ++q) r[q] = 0u;
#pragma unroll
        for (int c = 0; c < kAccs; ++c) {
            if (!((started >> c) & 1u)) continue;
            tc::ld_32x32b_x32(ta + (uint32_t)c * kTcN, t);
            tc::wait_ld();
#pragma unroll
            for (int q = 0; q < 32; ++q) r[q] = __float_as_uint(__uint_as_float(r[q]) + __uint_as_float(t[q]));
        }
        const int col = n_tile * kTcN + cb * 32;
        const int n = min(32, a.nu - col);
        if (row_ok && n > 0) store_row32<TQ>(Q + grow * a.nu + col, r, n);
        if (a.view_max && row_ok) {
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (q < n) amax = max(amax, r[q] & 0x7fffffffu);
        }
    }
    if (a.view_max) view_max_reduce(a.view_max, row_ok ? (int)(grow / a.nv) : -1, amax, lane);
    if (!ok || aborted) {
        if (tid == 0) atomicOr(a.status, kStatusTimeout);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::dealloc(tmem, kTmemCols);
}

// Weighted row w(k) = E F_cos as a double-float p + c (p = E F_hi rounded,
// c = the exact rounding error of p plus E F_lo); 0 outside [0, nu).
__device__ __forceinline__ void weighted(const float *__restrict__ Erow, const float *__restrict__ fh_row,
                                         const float *__restrict__ fl_row, int k, int nu, float &p, float &c)
{
    p = 0.0f;
    c = 0.0f;
    if (k >= 0 && k < nu) {
        const float x = __ldg(Erow + k), fh = __ldg(fh_row + k);
        p = x * fh;
        c = fmaf(x, __ldg(fl_row + k), fmaf(x, fh, -p));
    }
}

// First difference d(k) = w(k) - w(k-1) of rows [row0, row0 + nrows) split
// into `planes` BF16 terms, ws[t][r][k] (k < kpad; zero beyond nu).  The
// difference of the two double-floats is taken with a two-sum, then rounded
// once to FP32.
__global__ void __launch_bounds__(256)
    filter_split_kernel(const float *__restrict__ E, const float *__restrict__ fcos, const float *__restrict__ fcos_lo,
                        const float *__restrict__ sweight, __nv_bfloat16 *ws, int nu, int nv, int kpad, long long row0,
                        int nrows, int planes, long long plane)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int groups = kpad / 8;
    const long long r = idx / groups;
    const int k0 = (int)(idx - r * groups) * 8;
    if (r >= nrows) return;
    const long long grow = row0 + r;
    const int v = (int)(grow % nv);
    const float *Erow = E + grow * nu, *fh_row = fcos + (size_t)v * nu, *fl_row = fcos_lo + (size_t)v * nu;
    float p0, c0;
    weighted(Erow, fh_row, fl_row, k0 - 1, nu, p0, c0);
    // the 8 weighted elements k0 .. k0 + 7: float4 loads where the rows are 16-byte
    // aligned (nu a multiple of 4) and the group lies on the detector
    float pw[8], cw[8];
    if ((nu & 3) == 0 && k0 + 8 <= nu) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 x = __ldcs(reinterpret_cast<const float4 *>(Erow + k0) + h);
            const float4 fh = __ldg(reinterpret_cast<const float4 *>(fh_row + k0) + h);
            const float4 fl = __ldg(reinterpret_cast<const float4 *>(fl_row + k0) + h);
            const float xs[4] = {x.x, x.y, x.z, x.w}, hs[4] = {fh.x, fh.y, fh.z, fh.w}, ls[4] = {fl.x, fl.y, fl.z, fl.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                pw[4 * h + e] = xs[e] * hs[e];
                cw[4 * h + e] = fmaf(xs[e], ls[e], fmaf(xs[e], hs[e], -pw[4 * h + e]));
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) weighted(Erow, fh_row, fl_row, k0 + e, nu, pw[e], cw[e]);
    }
    if (sweight) {
        // short scan: the per-(view, column) redundancy weight, applied with F_cos
        const float *srow = sweight + (grow / nv) * nu;
        if (k0 > 0) df_scale(p0, c0, __ldg(srow + k0 - 1));
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (k0 + e < nu) df_scale(pw[e], cw[e], __ldg(srow + k0 + e));
    }
    uint32_t w[3][4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        uint16_t h[3][2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float p1 = pw[q + e], c1 = cw[q + e];
            const float s = p1 - p0, bb = s - p1;
            const float err = (p1 - (s - bb)) + (-p0 - bb);   // s + err = p1 - p0 exactly
            float rem = s + (err + (c1 - c0));
            p0 = p1;
            c0 = c1;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const __nv_bfloat16 b = __float2bfloat16_rn(rem);
                rem -= __bfloat162float(b);
                h[t][e] = *reinterpret_cast<const uint16_t *>(&b);
            }
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) w[t][q / 2] = (uint32_t)h[t][0] | ((uint32_t)h[t][1] << 16);
    }
#pragma unroll
    for (int t = 0; t < 3; ++t)   // unrolled: w stays in registers
        if (t < planes)
            *reinterpret_cast<uint4 *>(ws + t * plane + r * kpad + k0) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

uint16_t f2bf(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);   // round to nearest even (finite inputs)
    return (uint16_t)(u >> 16);
}
double bf2d(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// 3-D map [planes][rows][kpad] of BF16 whose box is box_planes planes of
// box_rows x 64 (the planes land one after another in shared memory).
int encode_bf16_3d(CUtensorMap *m, const void *base, uint64_t kpad, uint64_t rows, uint64_t planes, uint32_t box_rows,
                   uint32_t box_planes)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return IFDK_ERR_CUDA;
    const cuuint64_t dims[3] = {kpad, rows, planes};
    const cuuint64_t strides[2] = {kpad * 2, kpad * rows * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kTcK, box_rows, box_planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS
               ? IFDK_OK
               : IFDK_ERR_CUDA;
}

// Data planes of split s.
int data_planes(int terms) { return terms; }

// E, Q: views [view_begin, view_begin + view_count) (row 0 = row 0 of view view_begin)
template <typename TQ>
int launch_tc(ifdk_plan_s *p, const float *E, void *Q, int terms, void *ws, size_t ws_bytes, unsigned int *view_max,
              cudaStream_t stream, int view_begin, int view_count)
{
    const ifdk_geometry &g = p->g;
    const int kpad = p->tc_kpad, npad = p->tc_npad, planes = data_planes(terms);
    const long long rows = (long long)view_count * g.nv;
    const float *sweight = p->d_sweight ? p->d_sweight + (size_t)view_begin * g.nu : nullptr;
    const size_t row_bytes = (size_t)planes * kpad * 2;
    long long cap = (long long)(ws_bytes / row_bytes) / kTcM * kTcM;
    if (cap < kTcM) return IFDK_ERR_INVALID;
    if (cap > rows) cap = (rows + kTcM - 1) / kTcM * kTcM;
    if (cap > 65535LL * kTcM) cap = 65535LL * kTcM;
    CUtensorMap tmA, tmB;
    int rc = encode_bf16_3d(&tmA, ws, kpad, (uint64_t)cap, planes, kTcM, planes);
    if (rc == IFDK_OK) rc = encode_bf16_3d(&tmB, p->d_tsplit, kpad, npad, 3, kTcN, planes);
    if (rc != IFDK_OK) return rc;
    auto kern = filter_tc_kernel<TQ>;
    const size_t smem = tc_smem(planes);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return IFDK_ERR_CUDA;
    TcArgs a;
    a.Q = Q;
    a.status = p->d_status;
    a.wait_ns = p->wait_ns;
    a.nu = g.nu;
    a.nk = kpad / kTcK;
    a.npairs = terms == 3 ? 6 : (terms == 2 ? 3 : 1);
    a.planes = planes;
    a.view_max = view_max ? view_max + view_begin : nullptr;
    a.nv = g.nv;
    a.stages = tc_stages(planes);
    for (long long r0 = 0; r0 < rows; r0 += cap) {
        const int nr = (int)(rows - r0 < cap ? rows - r0 : cap);
        const long long threads = (long long)nr * (kpad / 8);
        filter_split_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(
            E, p->d_fcos, p->d_fcos_lo, sweight, static_cast<__nv_bfloat16 *>(ws), g.nu, g.nv, kpad, r0, nr,
            planes, cap * kpad);
        a.row0 = r0;
        a.nrows = nr;
        kern<<<dim3(npad / kTcN, (nr + kTcM - 1) / kTcM), kTcThreads, smem, stream>>>(tmA, tmB, a);
        if (cudaGetLastError() != cudaSuccess) return IFDK_ERR_CUDA;
    }
    return IFDK_OK;
}

}  // namespace

// Plan-time part: the Toeplitz matrix G[n][k] = g(n - k) for n < nu, k <= nu
// (g the running sum of the Ram-Lak taps, accumulated in FP64 from
// m = -(nu-1); g(-nu) = 0) as three BF16 planes, each the rounded remainder
// of the previous; zero elsewhere.
int plan_filter_tc(ifdk_plan_s *p)
{
    const int nu = p->g.nu;
    p->tc_kpad = (nu + 1 + kTcK - 1) / kTcK * kTcK;
    p->tc_npad = (nu + kTcN - 1) / kTcN * kTcN;
    std::vector<double> gsum(2 * (size_t)nu, 0.0);   // gsum[m + nu] = g(m), m in [-nu, nu - 1]
    for (int m = -nu + 1; m < nu; ++m) {
        const double h = m == 0 ? 0.25 : ((m & 1) ? -1.0 / (M_PI * M_PI * (double)m * m) : 0.0);
        gsum[m + nu] = gsum[m - 1 + nu] + h;
    }
    const size_t plane = (size_t)p->tc_npad * p->tc_kpad;
    std::vector<uint16_t> t(3 * plane, 0);
    for (int n = 0; n < nu; ++n)
        for (int k = 0; k <= nu; ++k) {
            double rem = gsum[n - k + nu];
            for (int q = 0; q < 3; ++q) {
                const uint16_t b = f2bf((float)rem);
                t[q * plane + (size_t)n * p->tc_kpad + k] = b;
                rem -= bf2d(b);
            }
        }
    if (cudaMalloc(&p->d_tsplit, t.size() * 2) != cudaSuccess) return IFDK_ERR_NOMEM;
    if (cudaMemcpy(p->d_tsplit, t.data(), t.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) return IFDK_ERR_CUDA;
    return IFDK_OK;
}

size_t filter_workspace_min(const ifdk_plan_s *p, int terms)
{
    return (size_t)data_planes(terms) * kTcM * p->tc_kpad * 2;
}

int launch_filter_tc(ifdk_plan_s *p, const float *E, void *Q, int q_dtype, int terms, void *ws, size_t ws_bytes,
                     cudaStream_t stream, unsigned int *view_max, int view_begin, int view_count)
{
    if (view_count < 0) view_count = p->g.np - view_begin;
    if (view_count == 0) return IFDK_OK;
    switch (q_dtype) {
    case IFDK_F32: return launch_tc<float>(p, E, Q, terms, ws, ws_bytes, view_max, stream, view_begin, view_count);
    case IFDK_F16: return launch_tc<__half>(p, E, Q, terms, ws, ws_bytes, view_max, stream, view_begin, view_count);
    default:
        return launch_tc<__nv_bfloat16>(p, E, Q, terms, ws, ws_bytes, view_max, stream, view_begin, view_count);
    }
}

}  // namespace ifdk
