// Plan creation, validation, status handling and the C-ABI entry points.
//
// The plan forms every geometric quantity in FP64 (Eq. 2 projection terms,
// FDK view weights, the F_cos table and the Ram-Lak taps of Algorithm 1) and
// casts the results to FP32 device tables: these are the only FP64 steps.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "ifdk_device.cuh"
#include "ifdk_internal.h"

namespace ifdk {

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Angular weight of view s: the caller's weight, or half the angular distance
// to the two neighbouring views (differences wrapped into (-pi, pi]).
double view_weight(const ifdk_plan_s &p, int s)
{
    const int n = p.g.np;
    if (!p.weights.empty()) return p.weights[s];
    if (n == 1) return 2.0 * M_PI;
    const double *a = p.angles.data();
    const double dp = std::remainder(a[(s + 1) % n] - a[s], 2.0 * M_PI);
    const double dm = std::remainder(a[s] - a[(s + n - 1) % n], 2.0 * M_PI);
    return 0.5 * (std::fabs(dp) + std::fabs(dm));
}

int validate(const ifdk_geometry *g)
{
    if (!g || g->np < 1 || g->nu < 2 || g->nv < 2 || g->nx < 1 || g->ny < 1 || g->nz < 1 || !g->angles)
        return IFDK_ERR_INVALID;
    if ((int64_t)g->nu * g->nv > (int64_t)1 << 30 || g->nx > 65536 || g->ny > 65536 || g->nz > 65536)
        return IFDK_ERR_INVALID;
    if (!finite_pos(g->sid) || !finite_pos(g->sdd) || !finite_pos(g->du) || !finite_pos(g->dv) ||
        !finite_pos(g->dx) || !finite_pos(g->dy) || !finite_pos(g->dz))
        return IFDK_ERR_GEOMETRY;
    if (!std::isfinite(g->off_u) || !std::isfinite(g->off_v) || !std::isfinite(g->vol_off_z))
        return IFDK_ERR_GEOMETRY;
    if (g->sdd <= g->sid) return IFDK_ERR_GEOMETRY;
    for (int s = 0; s < g->np; ++s) {
        if (!std::isfinite(g->angles[s])) return IFDK_ERR_GEOMETRY;
        if (g->view_weights && !std::isfinite(g->view_weights[s])) return IFDK_ERR_GEOMETRY;
    }
    // Every voxel must lie in front of the source plane with room to spare:
    // z = d + Y' >= d - r_xy, r_xy the largest distance of a voxel from the axis.
    const double hx = 0.5 * (g->nx - 1) * g->dx, hy = 0.5 * (g->ny - 1) * g->dy;
    if (std::sqrt(hx * hx + hy * hy) >= 0.9 * g->sid) return IFDK_ERR_GEOMETRY;
    return IFDK_OK;
}

// Host part of a plan: geometry copy, principal point, FP64 projection terms.
int init_host_plan(ifdk_plan_s *p, const ifdk_geometry *gin)
{
    p->g = *gin;
    p->angles.assign(gin->angles, gin->angles + gin->np);
    if (gin->view_weights) p->weights.assign(gin->view_weights, gin->view_weights + gin->np);
    p->g.angles = p->angles.data();
    p->g.view_weights = p->weights.empty() ? nullptr : p->weights.data();
    const ifdk_geometry &g = p->g;

    p->uc = (g.nu - 1) / 2.0 + g.off_u / g.du;
    p->vc = (g.nv - 1) / 2.0 + g.off_v / g.dv;
    const double two_vc = 2.0 * p->vc;
    p->two_vc = (int)std::lround(two_vc);
    p->fold_ok = std::fabs(two_vc - p->two_vc) < 1e-9 && g.vol_off_z == 0.0;
    // Half-turn view pairs: view s + np/2 is view s turned by pi, so voxel
    // (X, Y, Z) in view s and (-X, -Y, Z) in view s + np/2 project to the same
    // (u, v) with the same z (Mrot(b + pi) = -Mrot(b) in the XY plane).
    p->half_turn = g.np >= 2 && g.np % 2 == 0;
    for (int s = 0; p->half_turn && s < g.np / 2; ++s)
        p->half_turn = std::fabs(std::remainder(g.angles[s + g.np / 2] - g.angles[s] - M_PI, 2.0 * M_PI)) < 1e-9;
    // quarter turn: view s + np/4 is view s turned by pi/2 (with the half turn, so are
    // s + np/2 and s + 3np/4)
    p->quarter_turn = p->half_turn && g.np % 4 == 0;
    for (int s = 0; p->quarter_turn && s < g.np / 4; ++s)
        p->quarter_turn =
            std::fabs(std::remainder(g.angles[s + g.np / 4] - g.angles[s] - 0.5 * M_PI, 2.0 * M_PI)) < 1e-9;

    // Per-view projection terms, FP64 (Eq. 2: M1 . Mrot(b) . M0, multiplied out
    // in closed form and re-centred on the volume centre and principal point).
    // World point of centred voxel (i', j', k'): X = dx i', Y = -dy j', Z = -dz k' + off_z.
    // Mrot: X' = cos b X - sin b Y, Y' = sin b X + cos b Y; homogeneous z = d + Y'.
    // M1:   u - uc = D X' / (du z),  v - vc = D (-Z) / (dv z).
    p->terms.resize(g.np);
    for (int s = 0; s < g.np; ++s) {
        const double cb = std::cos(g.angles[s]), sb = std::sin(g.angles[s]);
        ViewTerms &t = p->terms[s];
        t.C0 = (float)(g.dx * sb);
        t.C1 = (float)(-g.dy * cb);
        t.C3 = (float)g.sid;
        t.A0 = (float)(g.sdd * g.dx * cb / g.du);
        t.A1 = (float)(g.sdd * g.dy * sb / g.du);
        t.A3 = 0.0f;
        t.B2 = (float)(g.sdd * g.dz / g.dv);
        t.B3 = (float)(-g.sdd * g.vol_off_z / g.dv);
        t.w = (float)(view_weight(*p, s) * g.sid * g.sdd / (2.0 * g.du));
        t.pad0 = t.pad1 = t.pad2 = 0.0f;
    }

    return IFDK_OK;
}

}  // namespace

int check_backproject_args(const ifdk_plan_s *p, const void *Q, int q_dtype, int view_begin, int view_count,
                           const float *vol)
{
    if (!p || !Q || !vol) return IFDK_ERR_INVALID;
    if (q_dtype != IFDK_F32 && q_dtype != IFDK_F16 && q_dtype != IFDK_BF16) return IFDK_ERR_INVALID;
    if (view_begin < 0 || view_count < 0 || view_begin > p->g.np || view_count > p->g.np - view_begin)
        return IFDK_ERR_INVALID;
    if (((uintptr_t)Q & 15) || ((uintptr_t)vol & 15)) return IFDK_ERR_ALIGNMENT;
    return IFDK_OK;
}

}  // namespace ifdk

using namespace ifdk;

extern "C" {

const char *ifdk_status_string(int code)
{
    switch (code) {
    case IFDK_OK: return "ok";
    case IFDK_ERR_INVALID: return "invalid argument";
    case IFDK_ERR_GEOMETRY: return "geometry not covered";
    case IFDK_ERR_ALIGNMENT: return "buffer not 16-byte aligned";
    case IFDK_ERR_CUDA: return "CUDA runtime error";
    case IFDK_ERR_TIMEOUT: return "bounded device wait ran out";
    case IFDK_ERR_NOMEM: return "out of memory";
    case IFDK_ERR_UNSUPPORTED: return "unsupported request";
    case IFDK_ERR_BOUNDS: return "checked build: access outside a kernel's window";
    default: return "unknown status";
    }
}

int ifdk_create(ifdk_plan *out, const ifdk_geometry *gin)
{
    if (!out) return IFDK_ERR_INVALID;
    *out = nullptr;
    int rc = validate(gin);
    if (rc != IFDK_OK) return rc;

    ifdk_plan_s *p = new (std::nothrow) ifdk_plan_s();
    if (!p) return IFDK_ERR_NOMEM;
    rc = init_host_plan(p, gin);
    if (rc != IFDK_OK) { delete p; return rc; }
    const ifdk_geometry &g = p->g;

    // Cosine weight D / sqrt(D^2 + a^2 + b^2) (hi / lo FP32 pair), Ram-Lak
    // taps h(m) and their running sum g(m) = sum_{j=-(nu-1)}^{m} h(j), FP64 then FP32.
    std::vector<float> fcos((size_t)g.nu * g.nv), fcos_lo(fcos.size()), taps(2 * (size_t)g.nu - 1),
        gsum(2 * (size_t)g.nu);
    for (int iv = 0; iv < g.nv; ++iv)
        for (int iu = 0; iu < g.nu; ++iu) {
            const double a = (iu - p->uc) * g.du, b = (iv - p->vc) * g.dv;
            const double f = g.sdd / std::sqrt(g.sdd * g.sdd + a * a + b * b);
            fcos[(size_t)iv * g.nu + iu] = (float)f;
            fcos_lo[(size_t)iv * g.nu + iu] = (float)(f - (double)(float)f);
        }
    for (int m = -(g.nu - 1); m <= g.nu - 1; ++m) {
        const double h = m == 0 ? 0.25 : (m % 2 == 0 ? 0.0 : -1.0 / (M_PI * M_PI * (double)m * m));
        taps[m + g.nu - 1] = (float)h;
    }
    double run = 0.0;   // g(-nu) = 0
    gsum[0] = 0.0f;
    for (int m = -(g.nu - 1); m <= g.nu - 1; ++m) {
        run += m == 0 ? 0.25 : (m % 2 == 0 ? 0.0 : -1.0 / (M_PI * M_PI * (double)m * m));
        gsum[m + g.nu] = (float)run;
    }

    if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return IFDK_ERR_CUDA; }
    bool ok = cudaMalloc(&p->d_terms, sizeof(ViewTerms) * g.np) == cudaSuccess &&
              cudaMalloc(&p->d_fcos, sizeof(float) * fcos.size()) == cudaSuccess &&
              cudaMalloc(&p->d_fcos_lo, sizeof(float) * fcos.size()) == cudaSuccess &&
              cudaMalloc(&p->d_taps, sizeof(float) * taps.size()) == cudaSuccess &&
              cudaMalloc(&p->d_gsum, sizeof(float) * gsum.size()) == cudaSuccess &&
              cudaMalloc(&p->d_status, sizeof(unsigned int)) == cudaSuccess;
    if (!ok) { cudaGetLastError(); ifdk_destroy(p); return IFDK_ERR_NOMEM; }
    ok = cudaMemcpy(p->d_terms, p->terms.data(), sizeof(ViewTerms) * g.np, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(p->d_fcos, fcos.data(), sizeof(float) * fcos.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(p->d_fcos_lo, fcos_lo.data(), sizeof(float) * fcos.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(p->d_taps, taps.data(), sizeof(float) * taps.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(p->d_gsum, gsum.data(), sizeof(float) * gsum.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(p->d_status, 0, sizeof(unsigned int)) == cudaSuccess;
    if (!ok) { cudaGetLastError(); ifdk_destroy(p); return IFDK_ERR_CUDA; }

    rc = plan_filter_tc(p);
    if (rc != IFDK_OK) { cudaGetLastError(); ifdk_destroy(p); return rc; }
    ok = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
        ok = cudaEventCreateWithFlags(&p->ev_copy[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->ev_bp[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) { cudaGetLastError(); ifdk_destroy(p); return IFDK_ERR_CUDA; }
    plan_backproject(p);
    plan_packed(p);
    rc = plan_view_split(p);
    if (rc != IFDK_OK) { ifdk_destroy(p); return rc; }
    *out = p;
    return IFDK_OK;
}

int ifdk_destroy(ifdk_plan p)
{
    if (!p) return IFDK_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device) cudaSetDevice(p->device);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    for (cudaEvent_t e : {p->ev_start, p->ev_copy[0], p->ev_copy[1], p->ev_bp[0], p->ev_bp[1]})
        if (e) cudaEventDestroy(e);
    cudaFree(p->d_terms);
    cudaFree(p->d_fcos);
    cudaFree(p->d_fcos_lo);
    cudaFree(p->d_taps);
    cudaFree(p->d_gsum);
    cudaFree(p->d_status);
    cudaFree(p->d_tsplit);
    cudaFree(p->d_split);
    cudaFree(p->d_sweight);
    if (dev >= 0 && dev != p->device) cudaSetDevice(dev);
    delete p;
    return IFDK_OK;
}

namespace {
// ifdk_filter and ifdk_filter_max; view_max: nullptr, or [np] zeroed on the stream
// E, Q hold views [view_begin, view_begin + view_count) (the whole scan: 0, np)
int filter_call(ifdk_plan p, const float *E, void *Q, int q_dtype, int split_terms, void *workspace,
                size_t workspace_bytes, float *view_max, void *stream, int view_begin = 0, int view_count = -1)
{
    if (!p || !E || !Q) return IFDK_ERR_INVALID;
    if (q_dtype != IFDK_F32 && q_dtype != IFDK_F16 && q_dtype != IFDK_BF16) return IFDK_ERR_INVALID;
    if (split_terms < 0 || split_terms > 3) return IFDK_ERR_INVALID;
    if (split_terms > 0) {
        if (!workspace || workspace_bytes < filter_workspace_min(p, split_terms)) return IFDK_ERR_INVALID;
        if (((uintptr_t)workspace & 127) || ((uintptr_t)E & 15) || ((uintptr_t)Q & 15)) return IFDK_ERR_ALIGNMENT;
    }
    if ((uintptr_t)view_max & 3) return IFDK_ERR_ALIGNMENT;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    unsigned int *vm = reinterpret_cast<unsigned int *>(view_max);
    if (vm && cudaMemsetAsync(vm, 0, sizeof(unsigned int) * p->g.np, (cudaStream_t)stream) != cudaSuccess)
        return IFDK_ERR_CUDA;
    if (split_terms == 0)
        return launch_filter(p, E, Q, q_dtype, 0, false, (cudaStream_t)stream, vm, view_begin, view_count);
    return launch_filter_tc(p, E, Q, q_dtype, split_terms, workspace, workspace_bytes, (cudaStream_t)stream, vm,
                            view_begin, view_count);
}
}  // namespace

int ifdk_filter(ifdk_plan p, const float *E, void *Q, int q_dtype, int split_terms, void *workspace,
                size_t workspace_bytes, void *stream)
{
    return filter_call(p, E, Q, q_dtype, split_terms, workspace, workspace_bytes, nullptr, stream);
}

int ifdk_filter_max(ifdk_plan p, const float *E, void *Q, int q_dtype, int split_terms, void *workspace,
                    size_t workspace_bytes, float *view_max, void *stream)
{
    if (!view_max) return IFDK_ERR_INVALID;
    return filter_call(p, E, Q, q_dtype, split_terms, workspace, workspace_bytes, view_max, stream);
}

int ifdk_filter_views(ifdk_plan p, const float *Ev, void *Qv, int q_dtype, int split_terms, int view_begin,
                      int view_count, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!p || view_begin < 0 || view_count < 0 || view_begin > p->g.np || view_count > p->g.np - view_begin)
        return IFDK_ERR_INVALID;
    if (view_count == 0) return IFDK_OK;
    return filter_call(p, Ev, Qv, q_dtype, split_terms, workspace, workspace_bytes, nullptr, stream, view_begin,
                       view_count);
}

int ifdk_filter_workspace_size(ifdk_plan p, int split_terms, size_t *min_bytes, size_t *preferred_bytes)
{
    if (!p || split_terms < 0 || split_terms > 3) return IFDK_ERR_INVALID;
    const size_t mn = split_terms ? filter_workspace_min(p, split_terms) : 0;
    const long long rows = (long long)p->g.np * p->g.nv;
    // preferred: every row in one launch, up to 1 GiB of split operands
    long long pref_rows = (rows + 127) / 128 * 128;
    if (mn && pref_rows * (long long)(mn / 128) > (1LL << 30)) pref_rows = std::max(128LL, (1LL << 30) / (long long)(mn / 128) / 128 * 128);
    if (min_bytes) *min_bytes = mn;
    if (preferred_bytes) *preferred_bytes = split_terms ? mn / 128 * (size_t)pref_rows : 0;
    return IFDK_OK;
}

int ifdk_filter_adjoint(ifdk_plan p, const float *G_Q, float *G_E, void *stream)
{
    if (!p || !G_Q || !G_E) return IFDK_ERR_INVALID;
    return launch_filter(p, G_Q, G_E, IFDK_F32, 0, true, (cudaStream_t)stream);
}

int ifdk_backproject(ifdk_plan p, const void *Q, int q_dtype, int view_begin, int view_count,
                     float *vol, void *stream)
{
    const int rc = check_backproject_args(p, Q, q_dtype, view_begin, view_count, vol);
    if (rc != IFDK_OK || view_count == 0) return rc;
    return launch_backproject(p, Q, q_dtype, view_begin, view_count, 0, p->g.np, vol, (cudaStream_t)stream);
}

int ifdk_backproject_views(ifdk_plan p, const void *Qv, int q_dtype, int view_begin, int view_count,
                           float *vol, void *stream)
{
    const int rc = check_backproject_args(p, Qv, q_dtype, view_begin, view_count, vol);
    if (rc != IFDK_OK || view_count == 0) return rc;
    return launch_backproject(p, Qv, q_dtype, view_begin, view_count, view_begin, view_count, vol,
                              (cudaStream_t)stream);
}

int ifdk_packed_size(ifdk_plan p, int q_dtype, size_t *view_bytes, int *rows, int *row_elems)
{
    if (!p) return IFDK_ERR_INVALID;
    if (q_dtype != IFDK_F32 && q_dtype != IFDK_F16 && q_dtype != IFDK_BF16) return IFDK_ERR_INVALID;
    if (!p->pk[q_dtype].path) return IFDK_ERR_UNSUPPORTED;
    if (view_bytes) *view_bytes = packed_view_bytes(p, q_dtype);
    if (rows) *rows = p->pk_rows;
    if (row_elems) *row_elems = p->pk_nu;
    return IFDK_OK;
}

int ifdk_pack_views(ifdk_plan p, const void *Q, int q_dtype, int view_count, void *Qp, void *stream)
{
    if (!p || !Q || !Qp) return IFDK_ERR_INVALID;
    if (q_dtype != IFDK_F32 && q_dtype != IFDK_F16 && q_dtype != IFDK_BF16) return IFDK_ERR_INVALID;
    if (view_count < 0 || view_count > p->g.np) return IFDK_ERR_INVALID;
    if (!p->pk[q_dtype].path) return IFDK_ERR_UNSUPPORTED;
    if (((uintptr_t)Q & 15) || ((uintptr_t)Qp & 15)) return IFDK_ERR_ALIGNMENT;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    return launch_pack(p, Q, q_dtype, view_count, Qp, (cudaStream_t)stream);
}

int ifdk_backproject_packed(ifdk_plan p, const void *Qp, int q_dtype, int view_begin, int view_count, float *vol,
                            void *stream)
{
    int rc = check_backproject_args(p, Qp, q_dtype, view_begin, view_count, vol);
    if (rc != IFDK_OK) return rc;
    if (!p->pk[q_dtype].path) return IFDK_ERR_UNSUPPORTED;
    if (view_count == 0) return IFDK_OK;
    return launch_backproject_packed(p, Qp, q_dtype, view_begin, view_count, 0, p->g.np, vol, (cudaStream_t)stream);
}

int ifdk_backproject_packed_pairs(ifdk_plan p, const void *Qp, int q_dtype, int view_begin, int view_count,
                                  int pair_begin, int pair_count, float *vol, void *stream)
{
    int rc = check_backproject_args(p, Qp, q_dtype, view_begin, view_count, vol);
    if (rc != IFDK_OK) return rc;
    if (!p->pk[q_dtype].path) return IFDK_ERR_UNSUPPORTED;
    const int npairs = (p->g.nz + 1) / 2;
    if (pair_begin < 0 || pair_count < 0 || pair_begin > npairs || pair_count > npairs - pair_begin)
        return IFDK_ERR_INVALID;
    if (view_count == 0 || pair_count == 0) return IFDK_OK;
    PkZRange zr;
    zr.pair0 = pair_begin;
    zr.pcount = pair_count;
    // the middle slice of an odd nz is its own mirror: stored once
    zr.nz_out = 2 * pair_count - ((p->g.nz & 1) && pair_begin + pair_count == npairs ? 1 : 0);
    return launch_backproject_packed(p, Qp, q_dtype, view_begin, view_count, 0, p->g.np, vol, (cudaStream_t)stream,
                                     zr);
}

int ifdk_backproject_packed_batch(ifdk_plan p, const void *Qpb, int q_dtype, int view_begin, int view_count,
                                  float *vol, void *stream)
{
    int rc = check_backproject_args(p, Qpb, q_dtype, view_begin, view_count, vol);
    if (rc != IFDK_OK) return rc;
    if (!p->pk[q_dtype].path) return IFDK_ERR_UNSUPPORTED;
    const int h = p->g.np / 2;
    if (p->g.np % 2 != 0 || view_begin + view_count > h) return IFDK_ERR_INVALID;
    if (view_count == 0) return IFDK_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    const cudaStream_t s = (cudaStream_t)stream;
    const int n = view_count, b = view_begin;
    // packed view q of the batch is view b + q for q < n, view b + h + q - n after
    if (p->use_half_turn && p->pk2[q_dtype].path) return launch_packed_pairs(p, Qpb, q_dtype, b, n, b, n, 2 * n, vol, s);
    rc = launch_backproject_packed(p, Qpb, q_dtype, b, n, b, 2 * n, vol, s);
    if (rc == IFDK_OK) rc = launch_backproject_packed(p, Qpb, q_dtype, b + h, n, b + h - n, 2 * n, vol, s);
    return rc;
}

int ifdk_backproject_packed_quads(ifdk_plan p, const void *Qpq, int q_dtype, int view_begin, int view_count,
                                  float *vol, void *stream)
{
    int rc = check_backproject_args(p, Qpq, q_dtype, view_begin, view_count, vol);
    if (rc != IFDK_OK) return rc;
    if (!p->pk[q_dtype].path) return IFDK_ERR_UNSUPPORTED;
    const int q4 = p->g.np / 4;
    if (p->g.np % 4 != 0 || view_begin + view_count > q4) return IFDK_ERR_INVALID;
    if (view_count == 0) return IFDK_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return IFDK_ERR_CUDA;
    const cudaStream_t s = (cudaStream_t)stream;
    const int n = view_count, b = view_begin;
    // packed view k n + q of the batch is view b + q + k np/4, k = 0..3
    if (p->use_quarter_turn && p->pk4[q_dtype].path) return launch_packed_quads(p, Qpq, q_dtype, b, n, b, n, 4 * n, vol, s);
    if (p->use_half_turn && p->pk2[q_dtype].path) {
        // slots 0 and 2, then slots 1 and 3, as half-turn pairs
        rc = launch_packed_pairs(p, Qpq, q_dtype, b, n, b, 2 * n, 4 * n, vol, s);
        if (rc == IFDK_OK) rc = launch_packed_pairs(p, Qpq, q_dtype, b + q4, n, b + q4 - n, 2 * n, 4 * n, vol, s);
        return rc;
    }
    for (int k = 0; k < 4 && rc == IFDK_OK; ++k)
        rc = launch_backproject_packed(p, Qpq, q_dtype, b + k * q4, n, b + k * q4 - k * n, 4 * n, vol, s);
    return rc;
}

int ifdk_set_view_pairing(ifdk_plan p, int enable)
{
    if (!p || enable < 0 || enable > 2) return IFDK_ERR_INVALID;
    p->use_half_turn = enable != 0;
    p->use_quarter_turn = enable == 2;
    return IFDK_OK;
}

namespace {
// Parker's redundancy weight of the ray (beta, gamma) of a short scan over
// [0, pi + 2 delta]: the ray (beta, gamma) is measured again as
// (beta + pi + 2 gamma, -gamma), and the two weights add to 1.
double parker_weight(double b, double gm, double d)
{
    if (b < 0.0 || b > M_PI + 2.0 * d) return 0.0;
    if (b < 2.0 * d - 2.0 * gm) {
        const double t = std::sin(M_PI / 4.0 * b / (d - gm));
        return t * t;
    }
    if (b <= M_PI - 2.0 * gm) return 1.0;
    const double t = std::sin(M_PI / 4.0 * (M_PI + 2.0 * d - b) / (d + gm));
    return t * t;
}
}  // namespace

int ifdk_set_short_scan(ifdk_plan p, int enable)
{
    if (!p || (enable != 0 && enable != 1)) return IFDK_ERR_INVALID;
    if (!enable) {
        cudaFree(p->d_sweight);
        p->d_sweight = nullptr;
        return IFDK_OK;
    }
    const ifdk_geometry &g = p->g;
    if (g.np < 3) return IFDK_ERR_GEOMETRY;
    for (int s = 1; s < g.np; ++s)
        if (!(g.angles[s] > g.angles[s - 1])) return IFDK_ERR_GEOMETRY;
    std::vector<double> gamma(g.nu);
    double gmax = 0.0;
    for (int u = 0; u < g.nu; ++u) {
        gamma[u] = std::atan((u - p->uc) * g.du / g.sdd);   // fan angle of column u
        gmax = std::max(gmax, std::fabs(gamma[u]));
    }
    const double range = g.angles[g.np - 1] - g.angles[0], delta = 0.5 * (range - M_PI);
    if (!(delta > gmax) || !(range < 2.0 * M_PI)) return IFDK_ERR_GEOMETRY;
    std::vector<float> w((size_t)g.np * g.nu);
    for (int s = 0; s < g.np; ++s)
        for (int u = 0; u < g.nu; ++u)   // 2 w: the full-scan FDK constant holds a 1/2 for the double cover
            w[(size_t)s * g.nu + u] = (float)(2.0 * parker_weight(g.angles[s] - g.angles[0], gamma[u], delta));
    if (!p->d_sweight && cudaMalloc(&p->d_sweight, sizeof(float) * w.size()) != cudaSuccess) {
        cudaGetLastError();
        return IFDK_ERR_NOMEM;
    }
    if (cudaMemcpy(p->d_sweight, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return IFDK_ERR_CUDA;
    return IFDK_OK;
}

int ifdk_set_view_split(ifdk_plan p, int max_splits)
{
    if (!p || max_splits < 0) return IFDK_ERR_INVALID;
    p->view_split_max = max_splits;
    return IFDK_OK;
}

int ifdk_view_split(ifdk_plan p, int q_dtype, int *splits)
{
    if (!p || !splits) return IFDK_ERR_INVALID;
    if (q_dtype != IFDK_F32 && q_dtype != IFDK_F16 && q_dtype != IFDK_BF16) return IFDK_ERR_INVALID;
    const bool quads = p->use_quarter_turn && p->pk4[q_dtype].path;
    const bool pairs = !quads && p->use_half_turn && p->pk2[q_dtype].path;
    const int nv = quads ? 4 : (pairs ? 2 : 1);
    *splits = packed_view_split(p, q_dtype, p->g.np / nv, nv);
    return IFDK_OK;
}

int ifdk_project(ifdk_plan p, const float *vol, float *P, int view_begin, int view_count, void *stream)
{
    if (!p || !vol || !P) return IFDK_ERR_INVALID;
    if (view_begin < 0 || view_count < 0 || view_begin > p->g.np || view_count > p->g.np - view_begin)
        return IFDK_ERR_INVALID;
    if (((uintptr_t)vol & 15) || ((uintptr_t)P & 15)) return IFDK_ERR_ALIGNMENT;
    if (view_count == 0) return IFDK_OK;
    return launch_project(p, vol, P, view_begin, view_count, (cudaStream_t)stream);
}

int ifdk_volume_slices(ifdk_plan p, const float *vol, void *out, int out_dtype, int k_begin, int k_count,
                       void *stream)
{
    if (!p) return IFDK_ERR_INVALID;
    if (out_dtype != IFDK_F32 && out_dtype != IFDK_F16 && out_dtype != IFDK_BF16) return IFDK_ERR_INVALID;
    if (k_begin < 0 || k_count < 0 || k_begin > p->g.nz || k_count > p->g.nz - k_begin) return IFDK_ERR_INVALID;
    if (k_count == 0) return IFDK_OK;
    if (!vol || !out) return IFDK_ERR_INVALID;
    if (((uintptr_t)vol & 15) || ((uintptr_t)out & 15)) return IFDK_ERR_ALIGNMENT;
    return launch_volume_slices(p, vol, out, out_dtype, k_begin, k_count, (cudaStream_t)stream);
}

int ifdk_last_device_status(ifdk_plan p, void *stream)
{
    if (!p) return IFDK_ERR_INVALID;
    unsigned int h = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, p->d_status, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(p->d_status, 0, sizeof(unsigned int), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return IFDK_ERR_CUDA;
    if (h & kStatusTimeout) return IFDK_ERR_TIMEOUT;
    if (h & kStatusBounds) return IFDK_ERR_BOUNDS;
    return IFDK_OK;
}

int ifdk_set_wait_limit(ifdk_plan p, uint64_t ns)
{
    if (!p) return IFDK_ERR_INVALID;
    p->wait_ns = ns ? ns : 2000000000ull;
    return IFDK_OK;
}

int ifdk_set_test_abort(ifdk_plan p, int group)
{
    if (!p) return IFDK_ERR_INVALID;
    p->test_abort_group = group < 0 ? -1 : group;
    return IFDK_OK;
}

int ifdk_wait_selftest(ifdk_plan p, uint64_t ns, void *stream)
{
    if (!p || ns == 0 || ns > 10000000000ull) return IFDK_ERR_INVALID;
    return launch_wait_selftest(p, ns, (cudaStream_t)stream);
}

static void fill_info(const ifdk_plan_s *p, const BpLaunch &b, int64_t *info)
{
    info[0] = b.path;
    info[1] = b.box_w;
    info[2] = b.box_h;
    info[3] = b.path ? kPairs : kGenZ;
    info[4] = b.path ? b.views : 1;
    info[5] = (int64_t)b.smem;
    info[6] = (int64_t)b.grid_x * b.grid_y;
    info[7] = p->g.np;
}

int ifdk_backproject_info(ifdk_plan p, int q_dtype, int64_t info[8])
{
    if (!p || !info) return IFDK_ERR_INVALID;
    if (q_dtype != IFDK_F32 && q_dtype != IFDK_F16 && q_dtype != IFDK_BF16) return IFDK_ERR_INVALID;
    fill_info(p, p->bp[q_dtype], info);
    return IFDK_OK;
}

// Launch of a full-range packed back-projection: quarter-turn quads or
// half-turn pairs when they apply (and are switched on).
static void fill_packed_info(const ifdk_plan_s *p, int q_dtype, int64_t *info)
{
    const bool quads = p->use_quarter_turn && p->pk4[q_dtype].path;
    const bool pairs = !quads && p->use_half_turn && p->pk2[q_dtype].path;
    const PkLaunch &b = quads ? p->pk4[q_dtype] : (pairs ? p->pk2[q_dtype] : p->pk[q_dtype]);
    info[0] = b.path ? (quads ? 4 : (pairs ? 2 : 1)) : 0;
    info[1] = b.bw;
    info[2] = b.box_h;
    info[3] = b.pairs;
    info[4] = b.stages;
    info[5] = (int64_t)b.smem;
    info[6] = (int64_t)b.grid_x * b.grid_y;
    info[7] = b.fold_w;
    info[8] = b.align;
    info[9] = p->pk_rows;
    info[10] = p->pk_nu;
    info[11] = p->pk_row0;
}

int ifdk_backproject_packed_info(ifdk_plan p, int q_dtype, int64_t info[12])
{
    if (!p || !info) return IFDK_ERR_INVALID;
    if (q_dtype != IFDK_F32 && q_dtype != IFDK_F16 && q_dtype != IFDK_BF16) return IFDK_ERR_INVALID;
    fill_packed_info(p, q_dtype, info);
    return IFDK_OK;
}

int ifdk_query_packed(const ifdk_geometry *g, int q_dtype, int view_pairing, int64_t info[12])
{
    if (!info || view_pairing < 0 || view_pairing > 2) return IFDK_ERR_INVALID;
    if (q_dtype != IFDK_F32 && q_dtype != IFDK_F16 && q_dtype != IFDK_BF16) return IFDK_ERR_INVALID;
    int rc = validate(g);
    if (rc != IFDK_OK) return rc;
    ifdk_plan_s tmp;
    rc = init_host_plan(&tmp, g);
    if (rc != IFDK_OK) return rc;
    plan_packed(&tmp);
    tmp.use_half_turn = view_pairing != 0;
    tmp.use_quarter_turn = view_pairing == 2;
    fill_packed_info(&tmp, q_dtype, info);
    return IFDK_OK;
}

int ifdk_query_rows(const ifdk_geometry *g, int view_begin, int view_count, int *row_begin, int *row_count)
{
    if (!row_begin || !row_count) return IFDK_ERR_INVALID;
    int rc = validate(g);
    if (rc != IFDK_OK) return rc;
    if (view_begin < 0 || view_count < 0 || view_begin > g->np || view_count > g->np - view_begin)
        return IFDK_ERR_INVALID;
    ifdk_plan_s tmp;
    rc = init_host_plan(&tmp, g);
    if (rc != IFDK_OK) return rc;
    const double cx = (g->nx - 1) / 2.0, cy = (g->ny - 1) / 2.0, cz = (g->nz - 1) / 2.0;
    double vmin = 1e300, vmax = -1e300;
    for (int s = view_begin; s < view_begin + view_count; ++s) {
        const double cb = std::cos(g->angles[s]), sb = std::sin(g->angles[s]);
        for (int q = 0; q < 4; ++q) {
            const double ip = (q & 1) ? cx : -cx, jp = (q & 2) ? cy : -cy;
            const double z = g->sid + g->dx * sb * ip - g->dy * cb * jp;   // homogeneous z at a column corner
            for (int e = 0; e < 2; ++e) {
                const double kp = e ? cz : -cz;
                const double v = tmp.vc + (g->sdd * g->dz * kp - g->sdd * g->vol_off_z) / (g->dv * z);
                vmin = std::min(vmin, v);
                vmax = std::max(vmax, v);
            }
        }
    }
    *row_begin = 0;
    *row_count = 0;
    if (view_count == 0) return IFDK_OK;
    // taps floor(v) and floor(v) + 1, one more row on each side for FP32 rounding
    const double lo = std::floor(vmin) - 1.0, hi = std::floor(vmax) + 2.0;
    if (hi < 0.0 || lo > g->nv - 1.0) return IFDK_OK;
    const int r0 = (int)std::max(lo, 0.0), r1 = (int)std::min(hi, g->nv - 1.0);
    *row_begin = r0;
    *row_count = r1 - r0 + 1;
    return IFDK_OK;
}

int ifdk_query_backproject(const ifdk_geometry *g, int q_dtype, int64_t info[10])
{
    if (!info) return IFDK_ERR_INVALID;
    if (q_dtype != IFDK_F32 && q_dtype != IFDK_F16 && q_dtype != IFDK_BF16) return IFDK_ERR_INVALID;
    int rc = validate(g);
    if (rc != IFDK_OK) return rc;
    ifdk_plan_s tmp;
    rc = init_host_plan(&tmp, g);
    if (rc != IFDK_OK) return rc;
    plan_backproject(&tmp);
    fill_info(&tmp, tmp.bp[q_dtype], info);
    info[8] = tmp.bp[q_dtype].fold_w;
    info[9] = tmp.bp[q_dtype].align;
    return IFDK_OK;
}

}  // extern "C"
