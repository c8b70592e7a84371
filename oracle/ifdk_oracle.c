/*
 * FP64 CPU oracle for the FDK hot path of iFDK (Chen, Wahib, Takizawa,
 * Takano, Matsuoka, "iFDK: A Scalable Framework for Instant High-resolution
 * Image Reconstruction", SC'19, arXiv 1909.02724).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA library: it is the plain
 * definition of what the hot path computes, written for a reader to check
 * against the paper by eye, with no blocking, fusion or reordering.
 *
 *   - geometry: projection matrix P_s = (M1 . Mrot(beta_s) . M0)[0:3]  (Sec. 3.2.1, Eq. 2,
 *     matrices M0, Mrot, M1 under the proof of Theorem 3)
 *   - filtering stage, Algorithm 1: pointwise cosine weight F_cos, then each
 *     detector row convolved with F_ramp (Ram-Lak, Kak & Slaney spatial form)
 *   - back-projection, Algorithm 2 (three inner products per voxel per view,
 *     f = 1/z, W_dis = f^2, (u,v) = (x,y) f), with interp2 of Algorithm 3
 *   - the exact adjoint of that back-projection (weighted bilinear splat)
 *
 * Readings where the paper is silent (all FP64, round-to-nearest, no FMA
 * contraction: built with -ffp-contract=off):
 *   - interp2 uses floor (not truncation) and reads 0 outside the detector;
 *   - F_ramp is h(0)=1/4, h(even != 0)=0, h(odd n)=-1/(pi^2 n^2), support
 *     |n| <= Nu-1, i.e. the exact linear (zero padded) convolution;
 *   - the FDK scale (Kak & Slaney, full-scan FDK) is folded into a per-view
 *     weight dbeta_s * d * D / (2 Du); dbeta_s is half the angular distance
 *     between the two neighbouring views (2 pi / Np for uniform angles);
 *   - the volume centre sits on the rotation axis, shifted along Z by
 *     vol_off_z; the principal point is ((Nu-1)/2 + off_u/Du, (Nv-1)/2 + off_v/Dv).
 *
 * Parity status: every function below is pinned by tests/test_oracle_*.py
 * against closed forms, invariants, brute force or an independent algorithm.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double sid, sdd;            /* d: source-isocenter, D: source-detector (mm) */
    int nu, nv;                 /* detector width / height (pixels) */
    double du, dv;              /* detector pitch (mm/pixel) */
    double off_u, off_v;        /* principal point offset from detector centre (mm) */
    int np;                     /* number of views */
    const double *angles;       /* np view angles (rad) */
    const double *view_weights; /* np angular weights (rad) or NULL for the spacing rule */
    int nx, ny, nz;             /* volume size (voxels) */
    double dx, dy, dz;          /* voxel pitch (mm/voxel) */
    double vol_off_z;           /* world Z of the volume centre (mm) */
} orc_geom;

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */

static void mat4_mul(const double a[16], const double b[16], double c[16])
{
    for (int r = 0; r < 4; ++r)
        for (int col = 0; col < 4; ++col) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += a[r * 4 + k] * b[k * 4 + col];
            c[r * 4 + col] = s;
        }
}

/* P_s = first three rows of M1 . Mrot(beta) . M0 (Eq. 2).  Row-major 3x4. */
void orc_projection_matrix(const orc_geom *g, int s, double P[12])
{
    const double beta = g->angles[s];
    const double cb = cos(beta), sb = sin(beta);
    /* M0 = diag(Dx,Dy,Dz,1) . [[1,0,0,-(Nx-1)/2],[0,-1,0,(Ny-1)/2],[0,0,-1,(Nz-1)/2],[0,0,0,1]],
       followed by the shift of the volume centre along Z. */
    const double scale0[16] = {g->dx, 0, 0, 0, 0, g->dy, 0, 0, 0, 0, g->dz, 0, 0, 0, 0, 1};
    const double flip0[16] = {1, 0, 0, -(g->nx - 1) / 2.0,
                              0, -1, 0, (g->ny - 1) / 2.0,
                              0, 0, -1, (g->nz - 1) / 2.0,
                              0, 0, 0, 1};
    const double shiftz[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, g->vol_off_z, 0, 0, 0, 1};
    /* Mrot = [[1,0,0,0],[0,0,-1,0],[0,1,0,d],[0,0,0,1]] . Rz(beta) */
    const double perm[16] = {1, 0, 0, 0, 0, 0, -1, 0, 0, 1, 0, g->sid, 0, 0, 0, 1};
    const double rz[16] = {cb, -sb, 0, 0, sb, cb, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    /* M1 = diag(1/Du,1/Dv,1,1) . [[D,0,uc*Du,0],[0,D,vc*Dv,0],[0,0,1,0],[0,0,0,1]] */
    const double ucdu = (g->nu - 1) * g->du / 2.0 + g->off_u;
    const double vcdv = (g->nv - 1) * g->dv / 2.0 + g->off_v;
    const double pitch1[16] = {1.0 / g->du, 0, 0, 0, 0, 1.0 / g->dv, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    const double proj1[16] = {g->sdd, 0, ucdu, 0, 0, g->sdd, vcdv, 0, 0, 0, 1, 0, 0, 0, 0, 1};

    double m0a[16], m0[16], mrot[16], m1[16], t[16], p4[16];
    mat4_mul(scale0, flip0, m0a);
    mat4_mul(shiftz, m0a, m0);
    mat4_mul(perm, rz, mrot);
    mat4_mul(pitch1, proj1, m1);
    mat4_mul(mrot, m0, t);
    mat4_mul(m1, t, p4);
    memcpy(P, p4, 12 * sizeof(double));
}

/* Angular weight of view s: user weight, or half the angular distance to the
   two neighbouring views (wrapped into (-pi, pi]); 2 pi for a single view. */
double orc_view_weight(const orc_geom *g, int s)
{
    if (g->view_weights) return g->view_weights[s];
    if (g->np == 1) return 2.0 * M_PI;
    const double *a = g->angles;
    int sp = (s + 1) % g->np, sm = (s + g->np - 1) % g->np;
    double dp = a[sp] - a[s], dm = a[s] - a[sm];
    dp = remainder(dp, 2.0 * M_PI);
    dm = remainder(dm, 2.0 * M_PI);
    return 0.5 * (fabs(dp) + fabs(dm));
}

/* FDK constant of view s: dbeta_s * d * D / (2 Du) (Kak & Slaney full-scan FDK). */
static double fdk_view_constant(const orc_geom *g, int s)
{
    return orc_view_weight(g, s) * g->sid * g->sdd / (2.0 * g->du);
}

/* ------------------------------------------------------------------ */
/* filtering stage (Algorithm 1)                                       */
/* ------------------------------------------------------------------ */

/* F_cos[v][u] = D / sqrt(D^2 + a^2 + b^2), a, b: pixel offset from the principal point (mm). */
void orc_cosine_weight(const orc_geom *g, double *fcos)
{
    const double uc = (g->nu - 1) / 2.0 + g->off_u / g->du;
    const double vc = (g->nv - 1) / 2.0 + g->off_v / g->dv;
    for (int iv = 0; iv < g->nv; ++iv)
        for (int iu = 0; iu < g->nu; ++iu) {
            double a = (iu - uc) * g->du, b = (iv - vc) * g->dv;
            fcos[(size_t)iv * g->nu + iu] = g->sdd / sqrt(g->sdd * g->sdd + a * a + b * b);
        }
}

/* Ram-Lak taps h(m) for m = -(n-1) .. n-1, stored at h[m + n - 1]. */
void orc_ramlak(int n, double *h)
{
    for (int m = -(n - 1); m <= n - 1; ++m) {
        double v;
        if (m == 0) v = 0.25;
        else if (m % 2 == 0) v = 0.0;
        else v = -1.0 / (M_PI * M_PI * (double)m * (double)m);
        h[m + n - 1] = v;
    }
}

/* Q[r][n] = sum_m h(n-m) * F_cos[v_r][m] * E[r][m] for the rows r of `rows`
   (row r is detector row rows_v[r] of some view); direct linear convolution. */
void orc_filter_rows_direct(const orc_geom *g, const double *E, const int *rows_v, int nrows,
                            double *Q)
{
    const int nu = g->nu;
    double *h = (double *)malloc(sizeof(double) * (2 * nu - 1));
    double *fcos = (double *)malloc(sizeof(double) * (size_t)nu * g->nv);
    double *w = (double *)malloc(sizeof(double) * nu);
    orc_ramlak(nu, h);
    orc_cosine_weight(g, fcos);
    for (int r = 0; r < nrows; ++r) {
        const double *e = E + (size_t)r * nu;
        const double *fc = fcos + (size_t)rows_v[r] * nu;
        for (int m = 0; m < nu; ++m) w[m] = e[m] * fc[m];
        double *q = Q + (size_t)r * nu;
        for (int n = 0; n < nu; ++n) {
            double s = 0.0;
            for (int m = 0; m < nu; ++m) s += h[n - m + nu - 1] * w[m];
            q[n] = s;
        }
    }
    free(h);
    free(fcos);
    free(w);
}

/* In-place iterative radix-2 complex FFT of length L (power of two);
   sign = -1 forward, +1 inverse (unnormalised). */
static void fft_radix2(double *re, double *im, int L, int sign)
{
    for (int i = 1, j = 0; i < L; ++i) {
        int bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= L; len <<= 1) {
        double ang = sign * 2.0 * M_PI / len;
        for (int i = 0; i < L; i += len)
            for (int k = 0; k < len / 2; ++k) {
                double wr = cos(ang * k), wi = sin(ang * k);
                double xr = re[i + k + len / 2], xi = im[i + k + len / 2];
                double tr = xr * wr - xi * wi, ti = xr * wi + xi * wr;
                re[i + k + len / 2] = re[i + k] - tr;
                im[i + k + len / 2] = im[i + k] - ti;
                re[i + k] += tr;
                im[i + k] += ti;
            }
    }
}

/* Same result as orc_filter_rows_direct, through the convolution theorem
   (Sec. 2.2.3): zero-padded length L >= 2 Nu, forward FFT of the weighted row
   and of the circularly placed taps, pointwise product, inverse FFT. */
void orc_filter_rows_fft(const orc_geom *g, const double *E, const int *rows_v, int nrows,
                         double *Q)
{
    const int nu = g->nu;
    int L = 1;
    while (L < 2 * nu) L <<= 1;
    double *h = (double *)malloc(sizeof(double) * (2 * nu - 1));
    double *fcos = (double *)malloc(sizeof(double) * (size_t)nu * g->nv);
    double *hr = (double *)calloc(L, sizeof(double)), *hi = (double *)calloc(L, sizeof(double));
    double *xr = (double *)malloc(sizeof(double) * L), *xi = (double *)malloc(sizeof(double) * L);
    orc_ramlak(nu, h);
    orc_cosine_weight(g, fcos);
    for (int m = 0; m < nu; ++m) hr[m] = h[m + nu - 1];             /* h(m), m >= 0 */
    for (int m = 1; m < nu; ++m) hr[L - m] = h[-m + nu - 1];        /* h(-m) */
    fft_radix2(hr, hi, L, -1);
    for (int r = 0; r < nrows; ++r) {
        const double *e = E + (size_t)r * nu;
        const double *fc = fcos + (size_t)rows_v[r] * nu;
        for (int m = 0; m < L; ++m) { xr[m] = 0.0; xi[m] = 0.0; }
        for (int m = 0; m < nu; ++m) xr[m] = e[m] * fc[m];
        fft_radix2(xr, xi, L, -1);
        for (int m = 0; m < L; ++m) {
            double a = xr[m] * hr[m] - xi[m] * hi[m];
            double b = xr[m] * hi[m] + xi[m] * hr[m];
            xr[m] = a;
            xi[m] = b;
        }
        fft_radix2(xr, xi, L, +1);
        for (int n = 0; n < nu; ++n) Q[(size_t)r * nu + n] = xr[n] / L;
    }
    free(h); free(fcos); free(hr); free(hi); free(xr); free(xi);
}

/* ------------------------------------------------------------------ */
/* back-projection (Algorithms 2 and 3) and its adjoint                */
/* ------------------------------------------------------------------ */

/* Q_s lookup that reads 0 outside the detector; rowmap (optional) maps
   detector row v of view s to a row of a sparse Q, or -1 if absent (then
   *missing is set). */
typedef struct {
    const double *Q;       /* dense [np][nv][nu] (rowmap == NULL) or sparse [rows][nu] */
    const int64_t *rowmap; /* [np][nv] or NULL */
    int nu, nv;
    int missing;
} qview;

static double tap(qview *q, int s, int iu, int iv)
{
    if (iu < 0 || iu >= q->nu || iv < 0 || iv >= q->nv) return 0.0;
    if (q->rowmap) {
        int64_t r = q->rowmap[(size_t)s * q->nv + iv];
        if (r < 0) { q->missing = 1; return 0.0; }
        return q->Q[(size_t)r * q->nu + iu];
    }
    return q->Q[((size_t)s * q->nv + iv) * q->nu + iu];
}

/* interp2 (Algorithm 3) with floor and zero outside the detector. */
static double interp2(qview *q, int s, double u, double v)
{
    if (!(u > -2.0 && u < q->nu + 1.0 && v > -2.0 && v < q->nv + 1.0)) return 0.0;
    double fu = floor(u), fv = floor(v);
    int iu = (int)fu, iv = (int)fv;
    double du = u - fu, dv = v - fv;
    double t1 = tap(q, s, iu, iv) * (1.0 - du) + tap(q, s, iu + 1, iv) * du;
    double t2 = tap(q, s, iu, iv + 1) * (1.0 - du) + tap(q, s, iu + 1, iv + 1) * du;
    return t1 * (1.0 - dv) + t2 * dv;
}

/* One voxel, all views in [s0, s0+ns), summed in view order (Algorithm 2). */
static double bp_voxel(const orc_geom *g, const double *P, const double *wfdk, qview *q,
                       int s0, int ns, int i, int j, int k)
{
    double acc = 0.0;
    for (int s = s0; s < s0 + ns; ++s) {
        const double *p = P + 12 * s;
        double x = p[0] * i + p[1] * j + p[2] * k + p[3];
        double y = p[4] * i + p[5] * j + p[6] * k + p[7];
        double z = p[8] * i + p[9] * j + p[10] * k + p[11];
        double f = 1.0 / z;
        double wdis = f * f;
        double u = x * f, v = y * f;
        acc += wfdk[s] * wdis * interp2(q, s, u, v);
    }
    return acc;
}

typedef struct {
    const orc_geom *g;
    const double *P, *wfdk;
    qview q;
    int s0, ns;
    double *vol;                 /* dense volume [nx][ny][nz] (k fastest) or NULL */
    const int64_t *vox;          /* sampled voxels (i,j,k) triples, or NULL */
    double *out;                 /* sampled outputs */
    int64_t count;               /* columns (dense) or voxels (sampled) */
    int64_t next;                /* work counter, guarded by lock */
    pthread_mutex_t lock;
} bp_job;

static int64_t grab(bp_job *jb, int64_t chunk, int64_t *end)
{
    pthread_mutex_lock(&jb->lock);
    int64_t b = jb->next;
    jb->next += chunk;
    pthread_mutex_unlock(&jb->lock);
    *end = b + chunk < jb->count ? b + chunk : jb->count;
    return b;
}

static void *bp_worker(void *arg)
{
    bp_job *jb = (bp_job *)arg;
    const orc_geom *g = jb->g;
    qview q = jb->q;
    int64_t b, e;
    if (jb->vol) {
        while ((b = grab(jb, 4, &e)) < jb->count)
            for (int64_t col = b; col < e; ++col) {
                int i = (int)(col / g->ny), j = (int)(col % g->ny);
                for (int k = 0; k < g->nz; ++k)
                    jb->vol[((size_t)i * g->ny + j) * g->nz + k] +=
                        bp_voxel(g, jb->P, jb->wfdk, &q, jb->s0, jb->ns, i, j, k);
            }
    } else {
        while ((b = grab(jb, 64, &e)) < jb->count)
            for (int64_t t = b; t < e; ++t)
                jb->out[t] = bp_voxel(g, jb->P, jb->wfdk, &q, jb->s0, jb->ns, (int)jb->vox[3 * t],
                                      (int)jb->vox[3 * t + 1], (int)jb->vox[3 * t + 2]);
    }
    pthread_mutex_lock(&jb->lock);
    if (q.missing) jb->q.missing = 1;
    pthread_mutex_unlock(&jb->lock);
    return NULL;
}

static void tables(const orc_geom *g, double *P, double *wfdk)
{
    for (int s = 0; s < g->np; ++s) {
        orc_projection_matrix(g, s, P + 12 * s);
        wfdk[s] = fdk_view_constant(g, s);
    }
}

static int run_bp(bp_job *jb, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    pthread_mutex_init(&jb->lock, NULL);
    jb->next = 0;
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, bp_worker, jb);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&jb->lock);
    return jb->q.missing ? -1 : 0;
}

/* vol[i][j][k] += sum over views [s0, s0+ns) (k fastest).  Q dense [np][nv][nu]. */
int orc_backproject(const orc_geom *g, const double *Q, int s0, int ns, double *vol, int nthreads)
{
    double *P = (double *)malloc(sizeof(double) * 12 * g->np);
    double *w = (double *)malloc(sizeof(double) * g->np);
    tables(g, P, w);
    bp_job jb;
    memset(&jb, 0, sizeof(jb));
    jb.g = g; jb.P = P; jb.wfdk = w; jb.s0 = s0; jb.ns = ns; jb.vol = vol;
    jb.q.Q = Q; jb.q.nu = g->nu; jb.q.nv = g->nv;
    jb.count = (int64_t)g->nx * g->ny;
    int rc = run_bp(&jb, nthreads);
    free(P);
    free(w);
    return rc;
}

/* out[t] = back-projection at voxel (vox[3t], vox[3t+1], vox[3t+2]) over all views.
   Q is dense (rowmap NULL) or sparse rows addressed through rowmap[np][nv]
   (-1 = row not supplied; returns -1 if such a row was needed). */
int orc_backproject_voxels(const orc_geom *g, const double *Q, const int64_t *rowmap,
                           const int64_t *vox, int64_t n, double *out, int nthreads)
{
    double *P = (double *)malloc(sizeof(double) * 12 * g->np);
    double *w = (double *)malloc(sizeof(double) * g->np);
    tables(g, P, w);
    bp_job jb;
    memset(&jb, 0, sizeof(jb));
    jb.g = g; jb.P = P; jb.wfdk = w; jb.s0 = 0; jb.ns = g->np;
    jb.q.Q = Q; jb.q.rowmap = rowmap; jb.q.nu = g->nu; jb.q.nv = g->nv;
    jb.vox = vox; jb.out = out; jb.count = n;
    int rc = run_bp(&jb, nthreads);
    free(P);
    free(w);
    return rc;
}

/* Marks in need[np][nv] every detector row that the bilinear taps of the
   given voxels touch (used to filter only those rows for sampled checks). */
void orc_rows_needed(const orc_geom *g, const int64_t *vox, int64_t n, unsigned char *need)
{
    double *P = (double *)malloc(sizeof(double) * 12 * g->np);
    for (int s = 0; s < g->np; ++s) orc_projection_matrix(g, s, P + 12 * s);
    for (int64_t t = 0; t < n; ++t) {
        int i = (int)vox[3 * t], j = (int)vox[3 * t + 1], k = (int)vox[3 * t + 2];
        for (int s = 0; s < g->np; ++s) {
            const double *p = P + 12 * s;
            double y = p[4] * i + p[5] * j + p[6] * k + p[7];
            double z = p[8] * i + p[9] * j + p[10] * k + p[11];
            double v = y / z;
            if (!(v > -2.0 && v < g->nv + 1.0)) continue;
            int iv = (int)floor(v);
            if (iv >= 0 && iv < g->nv) need[(size_t)s * g->nv + iv] = 1;
            if (iv + 1 >= 0 && iv + 1 < g->nv) need[(size_t)s * g->nv + iv + 1] = 1;
        }
    }
    free(P);
}

/* Adjoint of orc_backproject: Pout[s][v][u] += weight * vol(i,j,k) for every
   bilinear tap of every voxel, views [s0, s0+ns).  Threads split the views. */
typedef struct {
    const orc_geom *g;
    const double *P, *wfdk, *vol;
    double *out;
    int s0, ns, stride, first;
} proj_job;

static void splat(double *Qs, int nu, int nv, int iu, int iv, double val)
{
    if (iu < 0 || iu >= nu || iv < 0 || iv >= nv) return;
    Qs[(size_t)iv * nu + iu] += val;
}

static void *proj_worker(void *arg)
{
    proj_job *jb = (proj_job *)arg;
    const orc_geom *g = jb->g;
    for (int s = jb->s0 + jb->first; s < jb->s0 + jb->ns; s += jb->stride) {
        const double *p = jb->P + 12 * s;
        double *Qs = jb->out + (size_t)s * g->nv * g->nu;
        for (int i = 0; i < g->nx; ++i)
            for (int j = 0; j < g->ny; ++j)
                for (int k = 0; k < g->nz; ++k) {
                    double x = p[0] * i + p[1] * j + p[2] * k + p[3];
                    double y = p[4] * i + p[5] * j + p[6] * k + p[7];
                    double z = p[8] * i + p[9] * j + p[10] * k + p[11];
                    double f = 1.0 / z;
                    double u = x * f, v = y * f;
                    if (!(u > -2.0 && u < g->nu + 1.0 && v > -2.0 && v < g->nv + 1.0)) continue;
                    double val = jb->wfdk[s] * f * f * jb->vol[((size_t)i * g->ny + j) * g->nz + k];
                    double fu = floor(u), fv = floor(v);
                    int iu = (int)fu, iv = (int)fv;
                    double du = u - fu, dv = v - fv;
                    splat(Qs, g->nu, g->nv, iu, iv, val * (1.0 - du) * (1.0 - dv));
                    splat(Qs, g->nu, g->nv, iu + 1, iv, val * du * (1.0 - dv));
                    splat(Qs, g->nu, g->nv, iu, iv + 1, val * (1.0 - du) * dv);
                    splat(Qs, g->nu, g->nv, iu + 1, iv + 1, val * du * dv);
                }
    }
    return NULL;
}

int orc_project(const orc_geom *g, const double *vol, int s0, int ns, double *Pout, int nthreads)
{
    double *P = (double *)malloc(sizeof(double) * 12 * g->np);
    double *w = (double *)malloc(sizeof(double) * g->np);
    tables(g, P, w);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    proj_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].g = g; jobs[t].P = P; jobs[t].wfdk = w; jobs[t].vol = vol; jobs[t].out = Pout;
        jobs[t].s0 = s0; jobs[t].ns = ns; jobs[t].stride = nthreads; jobs[t].first = t;
        pthread_create(&th[t], NULL, proj_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(P);
    free(w);
    return 0;
}
