/*
 * FP64 brute-force oracle for compositional sparse-voxel rendering.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (DrivingVoxels, Sec. 3.4 and Algorithm 1 of the supplement):
 *   - one ray per pixel centre, r(tau) = o + tau d with |d| = 1 (Sec. 3.4);
 *   - each actor's oriented box is intersected with the ray in the actor's
 *     local frame, reached through the inverse of its pose (Sec. 3.4, Alg. 1);
 *   - the entry/exit distances are sorted to split [near, far] into a
 *     front-to-back sequence of background and actor intervals (Sec. 3.4);
 *   - inside each interval, the owning octree's voxels are composited front to
 *     back with the running state (C, D, T) carried across interval borders
 *     (Alg. 1), stopping once T < eps_stop;
 *   - per voxel segment: trilinear interpolation of the eight raw corner
 *     densities (Sec. 3.1), exponential-linear activation, midpoint numerical
 *     integration and alpha compositing (Sec. 3.4, formulas taken over from
 *     SVRaster), colour from SH coefficients (Sec. 3.1).
 *
 * The brute force is deliberate: every voxel of every octree is tested against
 * every ray, all clipped sub-segments are collected and sorted by
 * (t0, octree index, voxel index) and then composited.  There is no culling,
 * no tiling and no ordering trick.
 *
 * Readings where the paper delegates to SVRaster or is silent (each is also a
 * line of the design notes):
 *   explin(x) = x for x > 1.1, else 1.1 * exp(x / 1.1 - 1)  (C1 at 1.1);
 *   interpolation on raw values, activation after interpolation;
 *   K uniform midpoint samples on each clipped segment, tau = (l/K) sum sigma;
 *   alpha = 1 - exp(-tau); T <- T (1 - alpha); early stop checked after every
 *   segment; depth D = sum_k T_k alpha_k (t0 + t1) / 2 (not divided by alpha);
 *   colour = max(0, sum_lm Y_lm(g) k_lm + 0.5) with g the unit direction from
 *   the camera centre to the voxel centre in the octree's local frame;
 *   overlapping actor boxes: the box entered first owns the overlap;
 *   the garbled "D = 1" of Alg. 1's initial state is read as T = 1;
 *   the normal state N of Alg. 1 (Sec. 3.4: the pixel state sums voxel normals) is
 *   N = sum_k T_k alpha_k n_k with n the voxel's normal in world coordinates:
 *   minus the normalised gradient of the voxel's trilinear raw density at its
 *   centre, rotated by the octree's pose (zero where that gradient is zero).
 *
 * Backward: analytic reverse sweep of the same composite (chain rule through
 * C, D and alpha = 1 - T_final), accumulated into FP64 gradient arrays.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

#define ORC_ROLE_BG 0
#define ORC_ROLE_ACTOR 1

#define ORC_ACT_EXPLIN 0
#define ORC_ACT_IDENTITY 1

typedef struct {
    int64_t n_vox;
    int sh_degree;
    int role;            /* ORC_ROLE_BG or ORC_ROLE_ACTOR */
    int f64;             /* dens/sh element type: 0 = float, 1 = double */
    double center[3];
    double root_size;
    double clip_half[3]; /* actor clip box half extents (local frame) */
    const uint64_t* key; /* level << 57 | k << 38 | j << 19 | i */
    const void* dens;    /* [n][8], corner c at (c&1, c>>1&1, c>>2&1) */
    const void* sh;      /* [n][(deg+1)^2][3] */
} orc_octree;

typedef struct {
    double R[9]; /* row-major, local -> world: p_w = R p_l + t */
    double t[3];
} orc_pose;

typedef struct {
    int W, H;
    double fx, fy, cx, cy;
    orc_pose c2w; /* camera -> world, OpenCV axes (x right, y down, z forward) */
    double near_, far_;
} orc_camera;

typedef struct {
    int K;
    double eps_stop;
    int activation;
} orc_opts;

/* ------------------------------------------------------------------ */
/* scalar helpers                                                      */
/* ------------------------------------------------------------------ */

static double act_f(double x, int a) {
    if (a == ORC_ACT_IDENTITY) return x;
    return x > 1.1 ? x : 1.1 * exp(x / 1.1 - 1.0);
}

static double act_df(double x, int a) {
    if (a == ORC_ACT_IDENTITY) return 1.0;
    return x > 1.1 ? 1.0 : exp(x / 1.1 - 1.0);
}

static double get_dens(const orc_octree* oc, int64_t v, int c) {
    if (oc->f64) return ((const double*)oc->dens)[v * 8 + c];
    return (double)((const float*)oc->dens)[v * 8 + c];
}

static double get_sh(const orc_octree* oc, int64_t v, int lm, int ch) {
    int64_t nsh = (int64_t)(oc->sh_degree + 1) * (oc->sh_degree + 1);
    int64_t i = (v * nsh + lm) * 3 + ch;
    if (oc->f64) return ((const double*)oc->sh)[i];
    return (double)((const float*)oc->sh)[i];
}

/* Real spherical harmonics up to degree 3 of a unit vector (x, y, z), ordered
 * (l, m) = (0,0), (1,-1), (1,0), (1,1), (2,-2) ... (3,3), with the
 * normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) written out per term and
 * the Condon-Shortley sign on odd m. */
static void sh_basis(int deg, double x, double y, double z, double* Y) {
    const double pi = 3.14159265358979323846;
    Y[0] = sqrt(1.0 / (4.0 * pi));
    if (deg < 1) return;
    double k1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = -k1 * y;
    Y[2] = k1 * z;
    Y[3] = -k1 * x;
    if (deg < 2) return;
    double k2a = sqrt(15.0 / (4.0 * pi));
    double k2b = sqrt(5.0 / (16.0 * pi));
    double k2c = sqrt(15.0 / (16.0 * pi));
    Y[4] = k2a * x * y;
    Y[5] = -k2a * y * z;
    Y[6] = k2b * (3.0 * z * z - 1.0);
    Y[7] = -k2a * x * z;
    Y[8] = k2c * (x * x - y * y);
    if (deg < 3) return;
    double k3a = sqrt(35.0 / (32.0 * pi));
    double k3b = sqrt(105.0 / (4.0 * pi));
    double k3c = sqrt(21.0 / (32.0 * pi));
    double k3d = sqrt(7.0 / (16.0 * pi));
    double k3e = sqrt(105.0 / (16.0 * pi));
    Y[9] = -k3a * y * (3.0 * x * x - y * y);
    Y[10] = k3b * x * y * z;
    Y[11] = -k3c * y * (5.0 * z * z - 1.0);
    Y[12] = k3d * z * (5.0 * z * z - 3.0);
    Y[13] = -k3c * x * (5.0 * z * z - 1.0);
    Y[14] = k3e * z * (x * x - y * y);
    Y[15] = -k3a * x * (x * x - 3.0 * y * y);
}

/* voxel geometry from its key, in the octree's local frame */
static void voxel_box(const orc_octree* oc, int64_t v, double lo[3], double* s) {
    uint64_t key = oc->key[v];
    uint64_t m = (1ull << 19) - 1;
    int level = (int)((key >> 57) & 31ull);
    double ijk[3] = {(double)(key & m), (double)((key >> 19) & m), (double)((key >> 38) & m)};
    *s = ldexp(oc->root_size, -level);
    for (int a = 0; a < 3; ++a) lo[a] = oc->center[a] - 0.5 * oc->root_size + ijk[a] * (*s);
}

/* Ray / axis-aligned box [lo, hi]: returns 1 and the entry/exit distances when
 * the open chord has positive length. */
static int slab(const double o[3], const double d[3], const double lo[3], const double hi[3], double* t0,
                double* t1) {
    double a = -INFINITY, b = INFINITY;
    for (int k = 0; k < 3; ++k) {
        if (d[k] == 0.0) {
            if (o[k] < lo[k] || o[k] > hi[k]) return 0;
            continue;
        }
        double ta = (lo[k] - o[k]) / d[k];
        double tb = (hi[k] - o[k]) / d[k];
        if (ta > tb) {
            double tt = ta;
            ta = tb;
            tb = tt;
        }
        if (ta > a) a = ta;
        if (tb < b) b = tb;
    }
    if (!(a < b)) return 0;
    *t0 = a;
    *t1 = b;
    return 1;
}

/* local frame of a pose: q = R^T (p - t) */
static void to_local(const orc_pose* P, const double p[3], double q[3]) {
    double w[3] = {p[0] - P->t[0], p[1] - P->t[1], p[2] - P->t[2]};
    for (int r = 0; r < 3; ++r) q[r] = P->R[0 * 3 + r] * w[0] + P->R[1 * 3 + r] * w[1] + P->R[2 * 3 + r] * w[2];
}

static void dir_local(const orc_pose* P, const double d[3], double q[3]) {
    for (int r = 0; r < 3; ++r) q[r] = P->R[0 * 3 + r] * d[0] + P->R[1 * 3 + r] * d[1] + P->R[2 * 3 + r] * d[2];
}

static void pixel_ray(const orc_camera* cam, int u, int v, double o[3], double d[3]) {
    double dc[3] = {((double)u + 0.5 - cam->cx) / cam->fx, ((double)v + 0.5 - cam->cy) / cam->fy, 1.0};
    double n = 0.0;
    for (int r = 0; r < 3; ++r) {
        d[r] = cam->c2w.R[r * 3 + 0] * dc[0] + cam->c2w.R[r * 3 + 1] * dc[1] + cam->c2w.R[r * 3 + 2] * dc[2];
        n += d[r] * d[r];
    }
    n = sqrt(n);
    for (int r = 0; r < 3; ++r) {
        d[r] /= n;
        o[r] = cam->c2w.t[r];
    }
}

/* ------------------------------------------------------------------ */
/* interval partition (Sec. 3.4, Alg. 1)                               */
/* ------------------------------------------------------------------ */

typedef struct {
    double a, b;
    int oct;
} interval;

static int cmp_interval(const void* x, const void* y) {
    const interval* p = (const interval*)x;
    const interval* q = (const interval*)y;
    if (p->a < q->a) return -1;
    if (p->a > q->a) return 1;
    return (p->oct > q->oct) - (p->oct < q->oct);
}

/* Fills `own` with the intervals each octree owns along the ray: actors in
 * their boxes (first-entered owns overlaps), the background everywhere else in
 * [near, far].  Returns the number of intervals (sorted front to back). */
static int partition(const orc_octree* oct, int n_oct, const orc_pose* poses, const double o[3],
                     const double d[3], double tnear, double tfar, interval* own) {
    interval* hits = (interval*)malloc(sizeof(interval) * (size_t)(n_oct + 1));
    int nh = 0;
    for (int i = 0; i < n_oct; ++i) {
        if (oct[i].role != ORC_ROLE_ACTOR) continue;
        double ol[3], dl[3], lo[3], hi[3], a, b;
        to_local(&poses[i], o, ol);
        dir_local(&poses[i], d, dl);
        for (int k = 0; k < 3; ++k) {
            lo[k] = -oct[i].clip_half[k];
            hi[k] = oct[i].clip_half[k];
        }
        if (!slab(ol, dl, lo, hi, &a, &b)) continue;
        if (a < tnear) a = tnear;
        if (b > tfar) b = tfar;
        if (a < b) {
            hits[nh].a = a;
            hits[nh].b = b;
            hits[nh].oct = i;
            ++nh;
        }
    }
    qsort(hits, (size_t)nh, sizeof(interval), cmp_interval);
    int bg = -1;
    for (int i = 0; i < n_oct; ++i)
        if (oct[i].role == ORC_ROLE_BG) bg = i;
    int n = 0;
    double cur = tnear;
    for (int k = 0; k < nh; ++k) {
        double a = hits[k].a > cur ? hits[k].a : cur;
        if (!(hits[k].b > a)) continue; /* entirely inside an earlier box */
        if (a > cur && bg >= 0) {
            own[n].a = cur;
            own[n].b = a;
            own[n].oct = bg;
            ++n;
        }
        own[n].a = a;
        own[n].b = hits[k].b;
        own[n].oct = hits[k].oct;
        ++n;
        cur = hits[k].b;
    }
    if (tfar > cur && bg >= 0) {
        own[n].a = cur;
        own[n].b = tfar;
        own[n].oct = bg;
        ++n;
    }
    free(hits);
    return n;
}

/* ------------------------------------------------------------------ */
/* segments                                                            */
/* ------------------------------------------------------------------ */

typedef struct {
    double t0, t1;
    int oct;
    int64_t vox;
} segment;

typedef struct {
    segment* s;
    int64_t n, cap;
} seglist;

static int push_seg(seglist* L, double t0, double t1, int oct, int64_t vox) {
    if (L->n == L->cap) {
        int64_t nc = L->cap ? 2 * L->cap : 64;
        segment* ns = (segment*)realloc(L->s, sizeof(segment) * (size_t)nc);
        if (!ns) return ORC_ENOMEM;
        L->s = ns;
        L->cap = nc;
    }
    L->s[L->n].t0 = t0;
    L->s[L->n].t1 = t1;
    L->s[L->n].oct = oct;
    L->s[L->n].vox = vox;
    L->n++;
    return ORC_OK;
}

static int cmp_seg(const void* x, const void* y) {
    const segment* p = (const segment*)x;
    const segment* q = (const segment*)y;
    if (p->t0 < q->t0) return -1;
    if (p->t0 > q->t0) return 1;
    if (p->oct != q->oct) return (p->oct > q->oct) - (p->oct < q->oct);
    return (p->vox > q->vox) - (p->vox < q->vox);
}

/* All clipped voxel sub-segments along one pixel's ray, sorted front to back. */
static int gather(const orc_octree* oct, int n_oct, const orc_pose* poses, const orc_camera* cam, int u, int v,
                  seglist* L, double o[3], double d[3]) {
    L->n = 0;
    pixel_ray(cam, u, v, o, d);
    interval* own = (interval*)malloc(sizeof(interval) * (size_t)(2 * n_oct + 2));
    int n_own = partition(oct, n_oct, poses, o, d, cam->near_, cam->far_, own);
    for (int i = 0; i < n_oct; ++i) {
        double ol[3], dl[3];
        to_local(&poses[i], o, ol);
        dir_local(&poses[i], d, dl);
        for (int64_t vx = 0; vx < oct[i].n_vox; ++vx) {
            double lo[3], hi[3], s, t0, t1;
            voxel_box(&oct[i], vx, lo, &s);
            for (int k = 0; k < 3; ++k) hi[k] = lo[k] + s;
            if (!slab(ol, dl, lo, hi, &t0, &t1)) continue;
            for (int q = 0; q < n_own; ++q) {
                if (own[q].oct != i) continue;
                double a = t0 > own[q].a ? t0 : own[q].a;
                double b = t1 < own[q].b ? t1 : own[q].b;
                if (b > a && push_seg(L, a, b, i, vx) != ORC_OK) {
                    free(own);
                    return ORC_ENOMEM;
                }
            }
        }
    }
    free(own);
    qsort(L->s, (size_t)L->n, sizeof(segment), cmp_seg);
    return ORC_OK;
}

/* Per-segment quantities shared by the forward and the backward sweep. */
typedef struct {
    double tau, alpha, rgb[3], pre[3], mid, g[3];
    double dtau_ddens[8];
    double nrm[3]; /* voxel normal, world frame */
} seg_eval;

/* Gradient of the trilinear raw density of voxel v at its centre, in units of
 * one corner-density difference per voxel edge times 4: component a is the sum
 * of the four corners on the high side of axis a minus the four on the low
 * side.  (The true gradient is this divided by 4 * size; only its direction is
 * used.) */
static void dens_gradient(const orc_octree* oc, int64_t v, double g[3]) {
    for (int a = 0; a < 3; ++a) {
        g[a] = 0.0;
        for (int c = 0; c < 8; ++c) g[a] += ((c >> a) & 1) ? get_dens(oc, v, c) : -get_dens(oc, v, c);
    }
}

/* Voxel normal: n_local = -g / |g| (0 if g = 0), then n_world = R n_local. */
static void voxel_normal(const orc_octree* oc, const orc_pose* P, int64_t v, double n_loc[3], double n_world[3],
                         double* gnorm) {
    double g[3];
    dens_gradient(oc, v, g);
    double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    for (int a = 0; a < 3; ++a) n_loc[a] = gn > 0.0 ? -g[a] / gn : 0.0;
    for (int r = 0; r < 3; ++r)
        n_world[r] = P->R[r * 3 + 0] * n_loc[0] + P->R[r * 3 + 1] * n_loc[1] + P->R[r * 3 + 2] * n_loc[2];
    *gnorm = gn;
}

static void eval_segment(const orc_octree* oc, const orc_pose* P, const double o[3], const double d[3],
                         const segment* sg, const orc_opts* opt, seg_eval* e) {
    double ol[3], dl[3], lo[3], s;
    to_local(P, o, ol);
    dir_local(P, d, dl);
    voxel_box(oc, sg->vox, lo, &s);
    double l = sg->t1 - sg->t0;
    int K = opt->K;
    double sum = 0.0;
    for (int c = 0; c < 8; ++c) e->dtau_ddens[c] = 0.0;
    for (int k = 0; k < K; ++k) {
        double t = sg->t0 + ((double)k + 0.5) * l / (double)K;
        double x[3];
        for (int a = 0; a < 3; ++a) {
            x[a] = (ol[a] + t * dl[a] - lo[a]) / s;
            if (x[a] < 0.0) x[a] = 0.0;
            if (x[a] > 1.0) x[a] = 1.0;
        }
        double w[8], rho = 0.0;
        for (int c = 0; c < 8; ++c) {
            double wx = (c & 1) ? x[0] : 1.0 - x[0];
            double wy = (c & 2) ? x[1] : 1.0 - x[1];
            double wz = (c & 4) ? x[2] : 1.0 - x[2];
            w[c] = wx * wy * wz;
            rho += w[c] * get_dens(oc, sg->vox, c);
        }
        sum += act_f(rho, opt->activation);
        double da = act_df(rho, opt->activation) * l / (double)K;
        for (int c = 0; c < 8; ++c) e->dtau_ddens[c] += da * w[c];
    }
    e->tau = sum * l / (double)K;
    e->alpha = 1.0 - exp(-e->tau);
    e->mid = 0.5 * (sg->t0 + sg->t1);
    /* view direction: camera centre -> voxel centre, local frame */
    double g[3], gn = 0.0;
    for (int a = 0; a < 3; ++a) {
        g[a] = lo[a] + 0.5 * s - ol[a];
        gn += g[a] * g[a];
    }
    gn = sqrt(gn);
    for (int a = 0; a < 3; ++a) e->g[a] = gn > 0.0 ? g[a] / gn : 0.0;
    double Y[16];
    sh_basis(oc->sh_degree, e->g[0], e->g[1], e->g[2], Y);
    int nsh = (oc->sh_degree + 1) * (oc->sh_degree + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double c = 0.5;
        for (int lm = 0; lm < nsh; ++lm) c += Y[lm] * get_sh(oc, sg->vox, lm, ch);
        e->pre[ch] = c;
        e->rgb[ch] = c > 0.0 ? c : 0.0;
    }
    double n_loc[3], grad_norm;
    voxel_normal(oc, P, sg->vox, n_loc, e->nrm, &grad_norm);
}

/* ------------------------------------------------------------------ */
/* forward                                                             */
/* ------------------------------------------------------------------ */

typedef struct {
    const orc_octree* oct;
    int n_oct;
    const orc_pose* poses;
    const orc_camera* cam;
    const orc_opts* opt;
    int64_t n_pix;
    const int64_t* pix;
    double *rgb, *depth, *alpha, *normal;
    int32_t* n_seg;
    const double *g_rgb, *g_depth, *g_alpha, *g_normal;
    /* backward: per-thread records */
    int tid, n_threads;
    int status;
    struct grad_rec* rec;
    int64_t n_rec, cap_rec;
} job;

struct grad_rec {
    int oct;
    int64_t vox;
    double g_dens[8];
    double g_rgb[3];
    double pre[3];
    double g[3];
    double g_nrm[3]; /* dL/d(voxel normal, world frame) from this segment */
};

static int64_t pixel_index(const job* J, int64_t p) { return J->pix ? J->pix[p] : p; }

static void* fwd_worker(void* arg) {
    job* J = (job*)arg;
    seglist L = {0, 0, 0};
    for (int64_t p = J->tid; p < J->n_pix; p += J->n_threads) {
        int64_t q = pixel_index(J, p);
        int u = (int)(q % J->cam->W), v = (int)(q / J->cam->W);
        double o[3], d[3];
        if (gather(J->oct, J->n_oct, J->poses, J->cam, u, v, &L, o, d) != ORC_OK) {
            J->status = ORC_ENOMEM;
            break;
        }
        double C[3] = {0, 0, 0}, D = 0.0, T = 1.0, N[3] = {0, 0, 0};
        int32_t used = 0;
        for (int64_t k = 0; k < L.n; ++k) {
            seg_eval e;
            const segment* sg = &L.s[k];
            eval_segment(&J->oct[sg->oct], &J->poses[sg->oct], o, d, sg, J->opt, &e);
            double w = T * e.alpha;
            for (int ch = 0; ch < 3; ++ch) C[ch] += w * e.rgb[ch];
            for (int a = 0; a < 3; ++a) N[a] += w * e.nrm[a];
            D += w * e.mid;
            T *= (1.0 - e.alpha);
            ++used;
            if (T < J->opt->eps_stop) break;
        }
        for (int ch = 0; ch < 3; ++ch) J->rgb[p * 3 + ch] = C[ch];
        J->depth[p] = D;
        J->alpha[p] = 1.0 - T;
        if (J->n_seg) J->n_seg[p] = used;
        if (J->normal)
            for (int a = 0; a < 3; ++a) J->normal[p * 3 + a] = N[a];
    }
    free(L.s);
    return NULL;
}

static int check_inputs(const orc_octree* oct, int n_oct, const orc_camera* cam, const orc_opts* opt) {
    if (!oct || n_oct < 0 || !cam || !opt) return ORC_EINVAL;
    if (opt->K < 1 || cam->W < 0 || cam->H < 0) return ORC_EINVAL;
    for (int i = 0; i < n_oct; ++i)
        if (oct[i].sh_degree < 0 || oct[i].sh_degree > 3) return ORC_EINVAL;
    return ORC_OK;
}

static int run_jobs(job* base, int n_threads, void* (*fn)(void*), job** out) {
    if (n_threads < 1) n_threads = 1;
    job* J = (job*)calloc((size_t)n_threads, sizeof(job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!J || !th) {
        free(J);
        free(th);
        return ORC_ENOMEM;
    }
    for (int t = 0; t < n_threads; ++t) {
        J[t] = *base;
        J[t].tid = t;
        J[t].n_threads = n_threads;
    }
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, fn, &J[t]);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    int st = ORC_OK;
    for (int t = 0; t < n_threads; ++t)
        if (J[t].status != ORC_OK) st = J[t].status;
    if (out)
        *out = J;
    else
        free(J);
    return st;
}

/* Forward render of `n_pix` pixels (linear index v*W+u; pix == NULL means all
 * W*H pixels in order).  Outputs rgb[n][3], depth[n], alpha[n] and, if
 * non-NULL, the number of composited segments per pixel and the normal state
 * normal[n][3] (world frame). */
int orc_render(const orc_octree* oct, int n_oct, const orc_pose* poses, const orc_camera* cam, const orc_opts* opt,
               int64_t n_pix, const int64_t* pix, double* rgb, double* depth, double* alpha, int32_t* n_seg,
               int n_threads, double* normal) {
    int st = check_inputs(oct, n_oct, cam, opt);
    if (st != ORC_OK) return st;
    if (!pix) n_pix = (int64_t)cam->W * cam->H;
    job base;
    memset(&base, 0, sizeof(base));
    base.oct = oct;
    base.n_oct = n_oct;
    base.poses = poses;
    base.cam = cam;
    base.opt = opt;
    base.n_pix = n_pix;
    base.pix = pix;
    base.rgb = rgb;
    base.depth = depth;
    base.alpha = alpha;
    base.n_seg = n_seg;
    base.normal = normal;
    return run_jobs(&base, n_threads, fwd_worker, NULL);
}

/* ------------------------------------------------------------------ */
/* backward                                                            */
/* ------------------------------------------------------------------ */

static int push_rec(job* J, const struct grad_rec* r) {
    if (J->n_rec == J->cap_rec) {
        int64_t nc = J->cap_rec ? 2 * J->cap_rec : 256;
        struct grad_rec* nr = (struct grad_rec*)realloc(J->rec, sizeof(struct grad_rec) * (size_t)nc);
        if (!nr) return ORC_ENOMEM;
        J->rec = nr;
        J->cap_rec = nc;
    }
    J->rec[J->n_rec++] = *r;
    return ORC_OK;
}

static void* bwd_worker(void* arg) {
    job* J = (job*)arg;
    seglist L = {0, 0, 0};
    seg_eval* E = NULL;
    int64_t capE = 0;
    for (int64_t p = J->tid; p < J->n_pix; p += J->n_threads) {
        int64_t q = pixel_index(J, p);
        int u = (int)(q % J->cam->W), v = (int)(q / J->cam->W);
        double o[3], d[3];
        if (gather(J->oct, J->n_oct, J->poses, J->cam, u, v, &L, o, d) != ORC_OK) {
            J->status = ORC_ENOMEM;
            break;
        }
        if (L.n > capE) {
            free(E);
            capE = L.n;
            E = (seg_eval*)malloc(sizeof(seg_eval) * (size_t)capE);
            if (!E) {
                J->status = ORC_ENOMEM;
                break;
            }
        }
        /* forward sweep, remembering T before each segment */
        double T = 1.0;
        int64_t n = 0;
        double* Tb = (double*)malloc(sizeof(double) * (size_t)(L.n + 1));
        for (int64_t k = 0; k < L.n; ++k) {
            const segment* sg = &L.s[k];
            eval_segment(&J->oct[sg->oct], &J->poses[sg->oct], o, d, sg, J->opt, &E[k]);
            Tb[k] = T;
            T *= (1.0 - E[k].alpha);
            n = k + 1;
            if (T < J->opt->eps_stop) break;
        }
        double Tend = T;
        const double* gC = &J->g_rgb[p * 3];
        double gD = J->g_depth[p], gA = J->g_alpha[p];
        double gN[3] = {0, 0, 0};
        if (J->g_normal)
            for (int a = 0; a < 3; ++a) gN[a] = J->g_normal[p * 3 + a];
        /* reverse sweep: R = contribution of everything behind segment k */
        double RC[3] = {0, 0, 0}, RD = 0.0, RN[3] = {0, 0, 0};
        for (int64_t k = n - 1; k >= 0; --k) {
            const seg_eval* e = &E[k];
            double Tn = Tb[k] * (1.0 - e->alpha); /* T after segment k */
            double w = Tb[k] * e->alpha;
            double gtau = gA * Tend;
            for (int ch = 0; ch < 3; ++ch) gtau += gC[ch] * (Tn * e->rgb[ch] - RC[ch]);
            gtau += gD * (Tn * e->mid - RD);
            for (int a = 0; a < 3; ++a) gtau += gN[a] * (Tn * e->nrm[a] - RN[a]);
            struct grad_rec r;
            r.oct = L.s[k].oct;
            r.vox = L.s[k].vox;
            for (int c = 0; c < 8; ++c) r.g_dens[c] = gtau * e->dtau_ddens[c];
            for (int ch = 0; ch < 3; ++ch) {
                r.g_rgb[ch] = gC[ch] * w;
                r.pre[ch] = e->pre[ch];
                r.g[ch] = e->g[ch];
                r.g_nrm[ch] = gN[ch] * w;
            }
            if (push_rec(J, &r) != ORC_OK) {
                J->status = ORC_ENOMEM;
                break;
            }
            for (int ch = 0; ch < 3; ++ch) RC[ch] += w * e->rgb[ch];
            RD += w * e->mid;
            for (int a = 0; a < 3; ++a) RN[a] += w * e->nrm[a];
        }
        free(Tb);
        if (J->status != ORC_OK) break;
    }
    free(L.s);
    free(E);
    return NULL;
}

/* Gradients of L w.r.t. every corner density and SH coefficient, given dL/dC,
 * dL/dD and dL/dalpha for `n_pix` pixels (same pixel convention as
 * orc_render), and dL/dN (g_normal[n][3], world frame; NULL = zero).  d_dens[i]
 * ([n][8]) and d_sh[i] ([n][nsh][3]) are accumulated
 * into (callers zero them). */
int orc_backward(const orc_octree* oct, int n_oct, const orc_pose* poses, const orc_camera* cam,
                 const orc_opts* opt, int64_t n_pix, const int64_t* pix, const double* g_rgb, const double* g_depth,
                 const double* g_alpha, double* const* d_dens, double* const* d_sh, int n_threads,
                 const double* g_normal) {
    int st = check_inputs(oct, n_oct, cam, opt);
    if (st != ORC_OK) return st;
    if (!pix) n_pix = (int64_t)cam->W * cam->H;
    job base;
    memset(&base, 0, sizeof(base));
    base.oct = oct;
    base.n_oct = n_oct;
    base.poses = poses;
    base.cam = cam;
    base.opt = opt;
    base.n_pix = n_pix;
    base.pix = pix;
    base.g_rgb = g_rgb;
    base.g_depth = g_depth;
    base.g_alpha = g_alpha;
    base.g_normal = g_normal;
    if (n_threads < 1) n_threads = 1;
    job* J = NULL;
    st = run_jobs(&base, n_threads, bwd_worker, &J);
    if (J) {
        for (int t = 0; t < n_threads; ++t) {
            for (int64_t r = 0; st == ORC_OK && r < J[t].n_rec; ++r) {
                const struct grad_rec* g = &J[t].rec[r];
                const orc_octree* oc = &oct[g->oct];
                for (int c = 0; c < 8; ++c) d_dens[g->oct][g->vox * 8 + c] += g->g_dens[c];
                if (g->g_nrm[0] != 0.0 || g->g_nrm[1] != 0.0 || g->g_nrm[2] != 0.0) {
                    /* through the voxel normal: n_local = -g/|g|, n_world = R n_local */
                    double n_loc[3], n_w[3], gn, dn[3], dg[3];
                    voxel_normal(oc, &poses[g->oct], g->vox, n_loc, n_w, &gn);
                    if (gn > 0.0) {
                        const double* R = poses[g->oct].R;
                        for (int k = 0; k < 3; ++k)
                            dn[k] = R[0 * 3 + k] * g->g_nrm[0] + R[1 * 3 + k] * g->g_nrm[1] + R[2 * 3 + k] * g->g_nrm[2];
                        double nd = n_loc[0] * dn[0] + n_loc[1] * dn[1] + n_loc[2] * dn[2];
                        for (int a = 0; a < 3; ++a) dg[a] = -(dn[a] - n_loc[a] * nd) / gn;
                        for (int c = 0; c < 8; ++c)
                            for (int a = 0; a < 3; ++a)
                                d_dens[g->oct][g->vox * 8 + c] += ((c >> a) & 1) ? dg[a] : -dg[a];
                    }
                }
                double Y[16];
                sh_basis(oc->sh_degree, g->g[0], g->g[1], g->g[2], Y);
                int nsh = (oc->sh_degree + 1) * (oc->sh_degree + 1);
                for (int ch = 0; ch < 3; ++ch) {
                    if (!(g->pre[ch] > 0.0)) continue; /* clamp at zero */
                    for (int lm = 0; lm < nsh; ++lm) d_sh[g->oct][(g->vox * nsh + lm) * 3 + ch] += Y[lm] * g->g_rgb[ch];
                }
            }
            free(J[t].rec);
        }
        free(J);
    }
    return st;
}

/* Debug/test helper: the sorted segment list of one pixel (up to `cap`
 * entries).  Returns the total number of segments along the ray (including
 * any not processed because of early stopping), or -1 on error. */
int64_t orc_pixel_segments(const orc_octree* oct, int n_oct, const orc_pose* poses, const orc_camera* cam, int u,
                           int v, int64_t cap, double* t0, double* t1, int32_t* oct_idx, int64_t* vox_idx) {
    seglist L = {0, 0, 0};
    double o[3], d[3];
    if (gather(oct, n_oct, poses, cam, u, v, &L, o, d) != ORC_OK) return -1;
    for (int64_t k = 0; k < L.n && k < cap; ++k) {
        t0[k] = L.s[k].t0;
        t1[k] = L.s[k].t1;
        oct_idx[k] = L.s[k].oct;
        vox_idx[k] = L.s[k].vox;
    }
    int64_t n = L.n;
    free(L.s);
    return n;
}

/* Compositing weights of pixel (u, v): for every segment that the forward
 * composites (front to back, with the early stop), its octree, voxel and weight
 * w_k = T_k alpha_k.  A feature f per voxel renders as F = sum_k w_k f(vox_k)
 * (the RGB accumulation with the colour replaced by a feature, as used for
 * feature fields); fusing 2-D features into voxels sums w_k F_pixel per voxel.
 * Returns the number of composited segments (at most `cap` are written), or -1. */
int64_t orc_pixel_weights(const orc_octree* oct, int n_oct, const orc_pose* poses, const orc_camera* cam,
                          const orc_opts* opt, int u, int v, int64_t cap, int32_t* oct_idx, int64_t* vox_idx,
                          double* weight) {
    if (check_inputs(oct, n_oct, cam, opt) != ORC_OK) return -1;
    seglist L = {0, 0, 0};
    double o[3], d[3];
    if (gather(oct, n_oct, poses, cam, u, v, &L, o, d) != ORC_OK) return -1;
    double T = 1.0;
    int64_t n = 0;
    for (int64_t k = 0; k < L.n; ++k) {
        seg_eval e;
        const segment* sg = &L.s[k];
        eval_segment(&oct[sg->oct], &poses[sg->oct], o, d, sg, opt, &e);
        if (n < cap) {
            oct_idx[n] = sg->oct;
            vox_idx[n] = sg->vox;
            weight[n] = T * e.alpha;
        }
        ++n;
        T *= (1.0 - e.alpha);
        if (T < opt->eps_stop) break;
    }
    free(L.s);
    return n;
}

/* Test helper: the real SH basis values used by the oracle. */
void orc_sh_basis(int deg, double x, double y, double z, double* Y) { sh_basis(deg, x, y, z, Y); }
