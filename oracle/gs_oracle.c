/*
 * gs_oracle.c -- plain, slow CPU oracle of the differentiable 3D Gaussian Splatting rasterizer
 * that MAGS-SLAM's per-agent mapping (Sec. III-A, Eq. 4) and joint pose-Gaussian refinement
 * (Sec. III-C, Eq. 23) optimise through: render RGB, depth and alpha of anisotropic Gaussians
 * seen from world-to-camera poses (Sec. III-B, Eq. 15), and differentiate a loss with respect to
 * every Gaussian parameter and to a per-view pose delta (Sec. III-C, "per-keyframe pose deltas").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this file; it exists so
 * that the CUDA library can be checked against an independent, obviously-correct computation.
 * It shares no code, header or constant table with the CUDA sources.
 *
 * Structure (no blocking or fusion beyond the definition):
 *   1. projection of every (view, Gaussian) pair: an FP32 "decision chain" (the exact operation
 *      sequence both implementations agree on, because it decides culling, tile binning and key
 *      order) and an FP64 "value chain" (the same mathematics in double precision);
 *   2. binning: one key (global tile << 32 | float bits of camera depth) per touched tile, emitted
 *      in (view, Gaussian)-major, tile row-major order, then a stable sort (qsort on key plus
 *      emission index) and [start, end) ranges per global tile;
 *   3. forward, per pixel: walk the pixel's tile list front to back, taking the skip / stop
 *      decisions in FP32 and accumulating colour, depth and transmittance in FP64;
 *   4. backward, per pixel: re-walk the list, store the blended entries with their FP64 alpha and
 *      transmittance, and accumulate the adjoint in reverse order;
 *   5. projection backward and pose gradient in FP64, by the chain rule through steps 1's value
 *      chain.
 *
 * Readings of points the paper leaves open (pixel centres at +0.5, near plane, Jacobian clamp,
 * radius, tile rectangle, key tie-break, the FP32 exp used for alpha decisions, termination before
 * blending, unnormalised depth, background, RGB colour without spherical harmonics, left-perturbed
 * pose twist) are stated where they are used below.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math: every float operation
 * must round exactly once, and a*b+c must never be fused unless written as fmaf).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------------ */
/* FP32 exponential used for every alpha / scale decision.                                     */
/*                                                                                              */
/* Cody-Waite argument reduction x = k ln2 + r, |r| <= ln2/2, then the degree-7 Taylor          */
/* polynomial of e^r evaluated by Horner's rule with fused multiply-adds, then scaling by 2^k   */
/* through the exponent field.  ln2 is split as hi + lo with hi = ln2 rounded to a multiple of  */
/* 2^-16 (16 significant bits, so k*hi is exact for |k| < 2^8) and lo = ln2 - hi rounded to     */
/* float.  Coefficients are 1/n! rounded to float.  Inputs <= -87 return 0, inputs > 88 return   */
/* +inf.                                                                                        */
/* ------------------------------------------------------------------------------------------ */
static const float OG_LOG2E = 1.44269504088896340736f;
static const float OG_LN2_HI = 0.693145751953125f;            /* 45426 / 65536 */
static const float OG_LN2_LO = 1.42860682030941723212e-6f;    /* ln2 - 45426/65536 */

static float og_expf(float x)
{
    if (!(x > -87.0f)) return 0.0f;
    if (x > 88.0f) return INFINITY;
    float kf = rintf(x * OG_LOG2E);
    float r = fmaf(-kf, OG_LN2_HI, x);
    r = fmaf(-kf, OG_LN2_LO, r);
    float p = 1.0f / 5040.0f;                 /* 1/7! */
    p = fmaf(p, r, 1.0f / 720.0f);            /* 1/6! */
    p = fmaf(p, r, 1.0f / 120.0f);            /* 1/5! */
    p = fmaf(p, r, 1.0f / 24.0f);             /* 1/4! */
    p = fmaf(p, r, 1.0f / 6.0f);              /* 1/3! */
    p = fmaf(p, r, 0.5f);                     /* 1/2! */
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int k = (int)kf;
    union { uint32_t u; float f; } sc;
    sc.u = (uint32_t)(k + 127) << 23;
    return p * sc.f;
}

void og_expf_batch(const float *x, float *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = og_expf(x[i]);
}

/* ------------------------------------------------------------------------------------------ */
/* Problem description                                                                         */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t n_views, width, height, tile_w, tile_h;
    int32_t pad0;
    int64_t n_gauss;
    const int64_t *view_begin;       /* [V] first Gaussian row rendered by the view  */
    const int64_t *view_end;         /* [V] one past the last row                     */
    /* FP32 decision inputs */
    const float *mu_f, *ls_f, *q_f, *o_f;   /* [n,3] [n,3] [n,4] [n]             */
    const float *cam_f;                     /* [V,16]: R(9, row-major) t(3) fx fy cx cy */
    /* FP64 value inputs */
    const double *mu_d, *ls_d, *q_d, *o_d, *c_d;
    const double *cam_d;                    /* [V,16]                              */
    /* constants (FP32; the value chain uses the same numbers widened to double) */
    float near_plane, dilation, radius_sigmas, alpha_max, alpha_min, t_min;
    float bg[3];
    int32_t pad1;
    const uint8_t *tile_mask;        /* [G] or NULL: only these global tiles are rendered */
} og_problem;

typedef struct {
    og_problem p;
    int32_t V, W, H, tw, th, Tx, Ty;
    int64_t G, VN;
    int64_t *voff;                   /* [V+1] flattened (view, Gaussian) offsets */
    /* FP32 decision chain, per (view, Gaussian) */
    float *mx, *my, *cA, *cB, *cC, *z, *rad, *op;
    int32_t *rect;                   /* [VN,4] x0 x1 y0 y1 (x1, y1 exclusive) */
    uint32_t *touched;
    int8_t *clx, *cly;               /* Jacobian clamp decisions: -1, 0, +1 */
    /* FP64 value chain */
    double *mxd, *myd, *cAd, *cBd, *cCd, *zd;
    /* bins */
    int64_t K;
    uint64_t *keys;
    uint32_t *vals;
    uint32_t *ranges;                /* [G,2] */
} og_ctx;

static inline const float *camf(const og_ctx *c, int v) { return c->p.cam_f + 16 * (int64_t)v; }
static inline const double *camd(const og_ctx *c, int v) { return c->p.cam_d + 16 * (int64_t)v; }

static inline int og_view_of(const og_ctx *c, int64_t f)
{
    int lo = 0, hi = c->V - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (c->voff[mid] <= f) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* ------------------------------------------------------------------------------------------ */
/* 1a. FP32 decision chain of the EWA projection                                               */
/*                                                                                              */
/* p_c = R mu + t (world-to-camera); Sigma = Rq S S^T Rq^T with S = diag(exp(l)) (Eq. 19 form); */
/* Sigma_2 = J R Sigma R^T J^T + dilation I, computed as U U^T with U = (J R)(Rq S);            */
/* conic = Sigma_2^-1; mean2D = (fx x/z + cx, fy y/z + cy); radius = ceil(3 sqrt(lambda_max));   */
/* tile rectangle of the bounding square.  Every operation is one correctly rounded float op,    */
/* fmaf where written.                                                                           */
/* ------------------------------------------------------------------------------------------ */
static void og_project_f32(og_ctx *c, int v, int64_t gi, int64_t f)
{
    const og_problem *P = &c->p;
    const float *cm = camf(c, v);
    const float *R = cm, *t = cm + 9;
    const float fx = cm[12], fy = cm[13], cx = cm[14], cy = cm[15];
    const float mx = P->mu_f[3 * gi], my = P->mu_f[3 * gi + 1], mz = P->mu_f[3 * gi + 2];

    c->touched[f] = 0;
    c->rad[f] = 0.0f;
    c->rect[4 * f] = c->rect[4 * f + 1] = c->rect[4 * f + 2] = c->rect[4 * f + 3] = 0;
    c->clx[f] = c->cly[f] = 0;
    c->mx[f] = c->my[f] = c->cA[f] = c->cB[f] = c->cC[f] = c->z[f] = 0.0f;
    c->op[f] = P->o_f[gi];

    float xc = fmaf(R[0], mx, fmaf(R[1], my, fmaf(R[2], mz, t[0])));
    float yc = fmaf(R[3], mx, fmaf(R[4], my, fmaf(R[5], mz, t[1])));
    float zc = fmaf(R[6], mx, fmaf(R[7], my, fmaf(R[8], mz, t[2])));
    c->z[f] = zc;
    if (!(zc > P->near_plane)) return;                          /* near-plane cull */

    /* unit quaternion (w,x,y,z) */
    float qw = P->q_f[4 * gi], qx = P->q_f[4 * gi + 1], qy = P->q_f[4 * gi + 2], qz = P->q_f[4 * gi + 3];
    float n2 = fmaf(qw, qw, fmaf(qx, qx, fmaf(qy, qy, qz * qz)));
    if (!(n2 > 0.0f)) return;
    float inv = 1.0f / sqrtf(n2);
    float w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float Rq[9];
    Rq[0] = 1.0f - 2.0f * (yy + zz); Rq[1] = 2.0f * (xy - wz);        Rq[2] = 2.0f * (xz + wy);
    Rq[3] = 2.0f * (xy + wz);        Rq[4] = 1.0f - 2.0f * (xx + zz); Rq[5] = 2.0f * (yz - wx);
    Rq[6] = 2.0f * (xz - wy);        Rq[7] = 2.0f * (yz + wx);        Rq[8] = 1.0f - 2.0f * (xx + yy);
    float s0 = og_expf(P->ls_f[3 * gi]), s1 = og_expf(P->ls_f[3 * gi + 1]), s2 = og_expf(P->ls_f[3 * gi + 2]);
    float M[9];
    for (int j = 0; j < 3; ++j) {
        M[3 * j] = Rq[3 * j] * s0; M[3 * j + 1] = Rq[3 * j + 1] * s1; M[3 * j + 2] = Rq[3 * j + 2] * s2;
    }

    /* perspective Jacobian with the normalised coordinates clamped to 1.3x the half field of view */
    float iz = 1.0f / zc;
    float limx = (0.65f * (float)c->W) / fx;
    float limy = (0.65f * (float)c->H) / fy;
    float ux = xc * iz, uy = yc * iz;
    float tx = fminf(limx, fmaxf(-limx, ux));
    float ty = fminf(limy, fmaxf(-limy, uy));
    c->clx[f] = (int8_t)(ux < -limx ? -1 : (ux > limx ? 1 : 0));
    c->cly[f] = (int8_t)(uy < -limy ? -1 : (uy > limy ? 1 : 0));
    float J00 = fx * iz, J11 = fy * iz;
    float J02 = -((fx * tx) * iz), J12 = -((fy * ty) * iz);
    float Wm[6];
    for (int k = 0; k < 3; ++k) {
        Wm[k] = fmaf(J00, R[k], J02 * R[6 + k]);
        Wm[3 + k] = fmaf(J11, R[3 + k], J12 * R[6 + k]);
    }
    float U[6];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k)
            U[3 * r + k] = fmaf(Wm[3 * r], M[k], fmaf(Wm[3 * r + 1], M[3 + k], Wm[3 * r + 2] * M[6 + k]));
    float a = fmaf(U[0], U[0], fmaf(U[1], U[1], U[2] * U[2])) + P->dilation;
    float b = fmaf(U[0], U[3], fmaf(U[1], U[4], U[2] * U[5]));
    float cc = fmaf(U[3], U[3], fmaf(U[4], U[4], U[5] * U[5])) + P->dilation;
    float det = fmaf(a, cc, -(b * b));
    if (!(det > 0.0f)) return;                                   /* degenerate footprint */
    float A = cc / det, B = -b / det, C = a / det;
    float px = fmaf(fx, ux, cx), py = fmaf(fy, uy, cy);
    float mid = 0.5f * (a + cc);
    float disc = fmaf(mid, mid, -det);
    float lam = mid + sqrtf(fmaxf(0.0f, disc));
    float rf = ceilf(P->radius_sigmas * sqrtf(lam));
    float tw = (float)c->tw, th = (float)c->th;
    float Tx = (float)c->Tx, Ty = (float)c->Ty;
    float x0 = fminf(fmaxf(floorf((px - rf) / tw), 0.0f), Tx);
    float x1 = fminf(fmaxf(floorf((px + rf) / tw) + 1.0f, 0.0f), Tx);
    float y0 = fminf(fmaxf(floorf((py - rf) / th), 0.0f), Ty);
    float y1 = fminf(fmaxf(floorf((py + rf) / th) + 1.0f, 0.0f), Ty);
    c->mx[f] = px; c->my[f] = py; c->cA[f] = A; c->cB[f] = B; c->cC[f] = C;
    c->rad[f] = rf;
    if (!(x1 > x0) || !(y1 > y0)) return;                        /* off-screen */
    c->rect[4 * f] = (int32_t)x0; c->rect[4 * f + 1] = (int32_t)x1;
    c->rect[4 * f + 2] = (int32_t)y0; c->rect[4 * f + 3] = (int32_t)y1;
    c->touched[f] = (uint32_t)((int32_t)(x1 - x0) * (int32_t)(y1 - y0));
}

/* ------------------------------------------------------------------------------------------ */
/* 1b. FP64 value chain of the same projection, with every intermediate the backward needs.    */
/* The clamp of the Jacobian's normalised coordinates follows the FP32 decision.                */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    double pc[3], iz, ux, uy, tx, ty, limx, limy;
    double J00, J02, J11, J12;
    double Wm[6], qraw[4], qn, q[4], Rq[9], s[3], M[9], U[6];
    double a, b, c, det, A, B, C, px, py;
} og_p64;

static void og_project_f64(const og_ctx *c, int v, int64_t gi, int64_t f, og_p64 *o)
{
    const og_problem *P = &c->p;
    const double *cm = camd(c, v);
    const double *R = cm, *t = cm + 9;
    const double fx = cm[12], fy = cm[13], cx = cm[14], cy = cm[15];
    const double *mu = P->mu_d + 3 * gi;
    for (int r = 0; r < 3; ++r) o->pc[r] = R[3 * r] * mu[0] + R[3 * r + 1] * mu[1] + R[3 * r + 2] * mu[2] + t[r];
    for (int k = 0; k < 4; ++k) o->qraw[k] = P->q_d[4 * gi + k];
    o->qn = sqrt(o->qraw[0] * o->qraw[0] + o->qraw[1] * o->qraw[1] + o->qraw[2] * o->qraw[2] + o->qraw[3] * o->qraw[3]);
    for (int k = 0; k < 4; ++k) o->q[k] = o->qraw[k] / o->qn;
    double w = o->q[0], x = o->q[1], y = o->q[2], z = o->q[3];
    double *Rq = o->Rq;
    Rq[0] = 1 - 2 * (y * y + z * z); Rq[1] = 2 * (x * y - w * z);     Rq[2] = 2 * (x * z + w * y);
    Rq[3] = 2 * (x * y + w * z);     Rq[4] = 1 - 2 * (x * x + z * z); Rq[5] = 2 * (y * z - w * x);
    Rq[6] = 2 * (x * z - w * y);     Rq[7] = 2 * (y * z + w * x);     Rq[8] = 1 - 2 * (x * x + y * y);
    for (int k = 0; k < 3; ++k) o->s[k] = exp(P->ls_d[3 * gi + k]);
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) o->M[3 * j + k] = Rq[3 * j + k] * o->s[k];
    double zc = o->pc[2];
    o->iz = 1.0 / zc;
    o->ux = o->pc[0] / zc;
    o->uy = o->pc[1] / zc;
    o->limx = 0.65 * (double)c->W / fx;
    o->limy = 0.65 * (double)c->H / fy;
    o->tx = c->clx[f] < 0 ? -o->limx : (c->clx[f] > 0 ? o->limx : o->ux);
    o->ty = c->cly[f] < 0 ? -o->limy : (c->cly[f] > 0 ? o->limy : o->uy);
    o->J00 = fx / zc; o->J11 = fy / zc;
    o->J02 = -fx * o->tx / zc; o->J12 = -fy * o->ty / zc;
    for (int k = 0; k < 3; ++k) {
        o->Wm[k] = o->J00 * R[k] + o->J02 * R[6 + k];
        o->Wm[3 + k] = o->J11 * R[3 + k] + o->J12 * R[6 + k];
    }
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k)
            o->U[3 * r + k] = o->Wm[3 * r] * o->M[k] + o->Wm[3 * r + 1] * o->M[3 + k] + o->Wm[3 * r + 2] * o->M[6 + k];
    double dil = (double)P->dilation;
    o->a = o->U[0] * o->U[0] + o->U[1] * o->U[1] + o->U[2] * o->U[2] + dil;
    o->b = o->U[0] * o->U[3] + o->U[1] * o->U[4] + o->U[2] * o->U[5];
    o->c = o->U[3] * o->U[3] + o->U[4] * o->U[4] + o->U[5] * o->U[5] + dil;
    o->det = o->a * o->c - o->b * o->b;
    o->A = o->c / o->det; o->B = -o->b / o->det; o->C = o->a / o->det;
    o->px = fx * o->ux + cx;
    o->py = fy * o->uy + cy;
}

/* ------------------------------------------------------------------------------------------ */
/* 2. binning                                                                                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct { uint64_t key; uint64_t emit; uint32_t val; } og_item;

static int og_cmp(const void *pa, const void *pb)
{
    const og_item *a = (const og_item *)pa, *b = (const og_item *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->emit != b->emit) return a->emit < b->emit ? -1 : 1;
    return 0;
}

static uint32_t og_fbits(float x) { union { float f; uint32_t u; } c; c.f = x; return c.u; }

og_ctx *og_create(const og_problem *P)
{
    og_ctx *c = (og_ctx *)calloc(1, sizeof(og_ctx));
    c->p = *P;
    c->V = P->n_views; c->W = P->width; c->H = P->height; c->tw = P->tile_w; c->th = P->tile_h;
    c->Tx = (c->W + c->tw - 1) / c->tw; c->Ty = (c->H + c->th - 1) / c->th;
    c->G = (int64_t)c->V * c->Tx * c->Ty;
    c->voff = (int64_t *)malloc(sizeof(int64_t) * (c->V + 1));
    c->voff[0] = 0;
    for (int v = 0; v < c->V; ++v) c->voff[v + 1] = c->voff[v] + (P->view_end[v] - P->view_begin[v]);
    int64_t VN = c->VN = c->voff[c->V];
    c->mx = (float *)malloc(4 * VN); c->my = (float *)malloc(4 * VN); c->cA = (float *)malloc(4 * VN);
    c->cB = (float *)malloc(4 * VN); c->cC = (float *)malloc(4 * VN); c->z = (float *)malloc(4 * VN);
    c->rad = (float *)malloc(4 * VN); c->op = (float *)malloc(4 * VN);
    c->rect = (int32_t *)malloc(16 * VN); c->touched = (uint32_t *)malloc(4 * VN);
    c->clx = (int8_t *)malloc(VN); c->cly = (int8_t *)malloc(VN);
    c->mxd = (double *)malloc(8 * VN); c->myd = (double *)malloc(8 * VN); c->cAd = (double *)malloc(8 * VN);
    c->cBd = (double *)malloc(8 * VN); c->cCd = (double *)malloc(8 * VN); c->zd = (double *)malloc(8 * VN);

    for (int v = 0; v < c->V; ++v) {
        int64_t b = P->view_begin[v], n = P->view_end[v] - b;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            int64_t f = c->voff[v] + i;
            og_project_f32(c, v, b + i, f);
            og_p64 o;
            og_project_f64(c, v, b + i, f, &o);
            c->mxd[f] = o.px; c->myd[f] = o.py; c->cAd[f] = o.A; c->cBd[f] = o.B; c->cCd[f] = o.C;
            c->zd[f] = o.pc[2];
        }
    }

    /* emit keys in (view, Gaussian)-major, tile row-major order */
    int64_t K = 0;
    for (int64_t f = 0; f < VN; ++f) K += c->touched[f];
    c->K = K;
    og_item *items = (og_item *)malloc(sizeof(og_item) * (K > 0 ? K : 1));
    int64_t e = 0;
    for (int v = 0; v < c->V; ++v) {
        for (int64_t f = c->voff[v]; f < c->voff[v + 1]; ++f) {
            if (!c->touched[f]) continue;
            const int32_t *rc = c->rect + 4 * f;
            for (int ty = rc[2]; ty < rc[3]; ++ty)
                for (int tx = rc[0]; tx < rc[1]; ++tx) {
                    uint64_t g = (uint64_t)v * c->Tx * c->Ty + (uint64_t)ty * c->Tx + tx;
                    items[e].key = (g << 32) | og_fbits(c->z[f]);
                    items[e].emit = (uint64_t)e;
                    items[e].val = (uint32_t)f;
                    ++e;
                }
        }
    }
    qsort(items, (size_t)K, sizeof(og_item), og_cmp);
    c->keys = (uint64_t *)malloc(8 * (K > 0 ? K : 1));
    c->vals = (uint32_t *)malloc(4 * (K > 0 ? K : 1));
    for (int64_t k = 0; k < K; ++k) { c->keys[k] = items[k].key; c->vals[k] = items[k].val; }
    free(items);
    c->ranges = (uint32_t *)calloc((size_t)(2 * c->G), 4);
    for (int64_t k = 0; k < K; ++k) {
        uint64_t g = c->keys[k] >> 32;
        if (k == 0 || (c->keys[k - 1] >> 32) != g) c->ranges[2 * g] = (uint32_t)k;
        if (k == K - 1 || (c->keys[k + 1] >> 32) != g) c->ranges[2 * g + 1] = (uint32_t)(k + 1);
    }
    return c;
}

void og_destroy(og_ctx *c)
{
    if (!c) return;
    free(c->voff); free(c->mx); free(c->my); free(c->cA); free(c->cB); free(c->cC); free(c->z);
    free(c->rad); free(c->op); free(c->rect); free(c->touched); free(c->clx); free(c->cly);
    free(c->mxd); free(c->myd); free(c->cAd); free(c->cBd); free(c->cCd); free(c->zd);
    free(c->keys); free(c->vals); free(c->ranges); free(c);
}

int64_t og_num_keys(const og_ctx *c) { return c->K; }
int64_t og_num_pairs(const og_ctx *c) { return c->VN; }

/* FP32 projection outputs: mean2d [VN,2], conic [VN,3], depth [VN], radius [VN], rect [VN,4],
 * touched [VN]; FP64 mean2d/conic/depth into the *_d arrays (any pointer may be NULL). */
void og_get_projection(const og_ctx *c, float *mean2d, float *conic, float *depth, float *radius,
                       int32_t *rect, uint32_t *touched, double *mean2d_d, double *conic_d, double *depth_d)
{
    for (int64_t f = 0; f < c->VN; ++f) {
        if (mean2d) { mean2d[2 * f] = c->mx[f]; mean2d[2 * f + 1] = c->my[f]; }
        if (conic) { conic[3 * f] = c->cA[f]; conic[3 * f + 1] = c->cB[f]; conic[3 * f + 2] = c->cC[f]; }
        if (depth) depth[f] = c->z[f];
        if (radius) radius[f] = c->rad[f];
        if (rect) memcpy(rect + 4 * f, c->rect + 4 * f, 16);
        if (touched) touched[f] = c->touched[f];
        if (mean2d_d) { mean2d_d[2 * f] = c->mxd[f]; mean2d_d[2 * f + 1] = c->myd[f]; }
        if (conic_d) { conic_d[3 * f] = c->cAd[f]; conic_d[3 * f + 1] = c->cBd[f]; conic_d[3 * f + 2] = c->cCd[f]; }
        if (depth_d) depth_d[f] = c->zd[f];
    }
}

void og_get_bins(const og_ctx *c, uint64_t *keys, uint32_t *vals, uint32_t *ranges)
{
    if (keys) memcpy(keys, c->keys, 8 * c->K);
    if (vals) memcpy(vals, c->vals, 4 * c->K);
    if (ranges) memcpy(ranges, c->ranges, 8 * c->G);
}

/* ------------------------------------------------------------------------------------------ */
/* 3./4. per-pixel compositing                                                                 */
/*                                                                                              */
/* Pixel (x, y) samples (x + 0.5, y + 0.5).  For each list entry, in order:                     */
/*   sigma = 1/2 (A dx^2 + C dy^2) + B dx dy,  d = pixel - mean2D;   skip if sigma < 0;          */
/*   alpha = min(alpha_max, o exp(-sigma));   skip if alpha < alpha_min;                         */
/*   T' = T (1 - alpha);  if T' < t_min the pixel stops and this entry is NOT blended;           */
/*   C += c alpha T,  D += z alpha T,  T = T'.                                                   */
/* Outputs: rgb = C + T_final bg, depth D (unnormalised), alpha = 1 - T_final, T_final, and      */
/* last = 1 + list position (relative to the tile range start) of the last blended entry.       */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    uint32_t f;
    uint8_t capped;
    double alpha, T, G, dx, dy;
} og_entry;

/* walks one pixel's list; fills entries (may be NULL) and returns the count of blended ones */
static int64_t og_walk(const og_ctx *c, int64_t g, int px_i, int py_i, og_entry *ent, double *rgb,
                       double *depth, double *Tfin, int32_t *last, int64_t *pairs)
{
    const og_problem *P = &c->p;
    uint32_t s = c->ranges[2 * g], e = c->ranges[2 * g + 1];
    float pxf = (float)px_i + 0.5f, pyf = (float)py_i + 0.5f;
    double pxd = (double)px_i + 0.5, pyd = (double)py_i + 0.5;
    float T32 = 1.0f;
    double T = 1.0, C[3] = {0, 0, 0}, D = 0.0;
    int64_t n = 0, np = 0;
    int32_t lst = 0;
    for (uint32_t j = s; j < e; ++j) {
        uint32_t f = c->vals[j];
        ++np;
        float dx = pxf - c->mx[f], dy = pyf - c->my[f];
        float q = fmaf(c->cA[f] * dx, dx, (c->cC[f] * dy) * dy);
        float sg = fmaf(c->cB[f] * dx, dy, 0.5f * q);
        if (sg < 0.0f) continue;
        float araw = c->op[f] * og_expf(-sg);
        int capped = araw > P->alpha_max;
        float a32 = capped ? P->alpha_max : araw;
        if (a32 < P->alpha_min) continue;
        float Tn = T32 * (1.0f - a32);
        if (Tn < P->t_min) break;
        /* FP64 values */
        int64_t gi;
        {
            int v = og_view_of(c, f);
            gi = P->view_begin[v] + (f - c->voff[v]);
        }
        double ddx = pxd - c->mxd[f], ddy = pyd - c->myd[f];
        double sgd = 0.5 * (c->cAd[f] * ddx * ddx + c->cCd[f] * ddy * ddy) + c->cBd[f] * ddx * ddy;
        double G = exp(-sgd);
        double ad = capped ? (double)P->alpha_max : P->o_d[gi] * G;
        for (int ch = 0; ch < 3; ++ch) C[ch] += P->c_d[3 * gi + ch] * ad * T;
        D += c->zd[f] * ad * T;
        if (ent) {
            ent[n].f = f; ent[n].capped = (uint8_t)capped; ent[n].alpha = ad; ent[n].T = T;
            ent[n].G = G; ent[n].dx = ddx; ent[n].dy = ddy;
        }
        ++n;
        T *= (1.0 - ad);
        T32 = Tn;
        lst = (int32_t)(j - s + 1);
    }
    if (rgb) for (int ch = 0; ch < 3; ++ch) rgb[ch] = C[ch] + T * (double)P->bg[ch];
    if (depth) *depth = D;
    if (Tfin) *Tfin = T;
    if (last) *last = lst;
    if (pairs) *pairs = np;
    return n;
}

/* rgb [V,3,H,W], depth/alpha/final_T [V,H,W] (FP64), last [V,H,W]; returns the number of
 * (pixel, list entry) pairs evaluated up to and including each pixel's stopping entry. */
int64_t og_forward(const og_ctx *c, double *rgb, double *depth, double *alpha, double *final_T, int32_t *last)
{
    const int64_t HW = (int64_t)c->W * c->H;
    int64_t total_pairs = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : total_pairs)
    for (int64_t g = 0; g < c->G; ++g) {
        if (c->p.tile_mask && !c->p.tile_mask[g]) continue;
        int v = (int)(g / ((int64_t)c->Tx * c->Ty));
        int tl = (int)(g % ((int64_t)c->Tx * c->Ty));
        int tx = tl % c->Tx, ty = tl / c->Tx;
        for (int yy = ty * c->th; yy < (ty + 1) * c->th && yy < c->H; ++yy)
            for (int xx = tx * c->tw; xx < (tx + 1) * c->tw && xx < c->W; ++xx) {
                double col[3], D, T;
                int32_t l;
                int64_t np;
                og_walk(c, g, xx, yy, NULL, col, &D, &T, &l, &np);
                int64_t pix = (int64_t)yy * c->W + xx;
                for (int ch = 0; ch < 3; ++ch) if (rgb) rgb[((int64_t)v * 3 + ch) * HW + pix] = col[ch];
                if (depth) depth[(int64_t)v * HW + pix] = D;
                if (alpha) alpha[(int64_t)v * HW + pix] = 1.0 - T;
                if (final_T) final_T[(int64_t)v * HW + pix] = T;
                if (last) last[(int64_t)v * HW + pix] = l;
                total_pairs += np;
            }
    }
    return total_pairs;
}

/* ------------------------------------------------------------------------------------------ */
/* 4. backward compositing: per (view, Gaussian) gradients of the 2-D quantities               */
/* g2d [VN,10] = dL/d(mean_x, mean_y, conic_A, conic_B, conic_C, opacity, depth, r, g, b).      */
/* ------------------------------------------------------------------------------------------ */
#define OG_ACC(dst, val)                 \
    do {                                 \
        double v_ = (val);               \
        if (shared_acc) {                \
            _Pragma("omp atomic")        \
            (dst) += v_;                 \
        } else {                         \
            (dst) += v_;                 \
        }                                \
    } while (0)

static void og_backward_2d(const og_ctx *c, const double *g_rgb, const double *g_depth, const double *g_alpha,
                           double *g2d)
{
    const og_problem *P = &c->p;
    const int64_t HW = (int64_t)c->W * c->H;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    /* one accumulator per thread, unless that would take more than 2 GB; then one shared
     * accumulator with atomic adds (only the FP64 summation order differs) */
    const char *force = getenv("GS_ORACLE_SHARED_ACC");
    const int shared_acc = (force && force[0] == '1') || (double)nthreads * (double)c->VN * 80.0 > 2e9;
    double *buf = (double *)calloc((size_t)(shared_acc ? 1 : nthreads) * c->VN * 10, sizeof(double));
    int64_t maxlen = 1;
    for (int64_t g = 0; g < c->G; ++g) {
        int64_t l = (int64_t)c->ranges[2 * g + 1] - c->ranges[2 * g];
        if (l > maxlen) maxlen = l;
    }
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *acc = buf + (size_t)(shared_acc ? 0 : tid) * c->VN * 10;
        og_entry *ent = (og_entry *)malloc(sizeof(og_entry) * maxlen);
#pragma omp for schedule(dynamic, 4)
        for (int64_t g = 0; g < c->G; ++g) {
            if (P->tile_mask && !P->tile_mask[g]) continue;
            int v = (int)(g / ((int64_t)c->Tx * c->Ty));
            int tl = (int)(g % ((int64_t)c->Tx * c->Ty));
            int tx = tl % c->Tx, ty = tl / c->Tx;
            for (int yy = ty * c->th; yy < (ty + 1) * c->th && yy < c->H; ++yy)
                for (int xx = tx * c->tw; xx < (tx + 1) * c->tw && xx < c->W; ++xx) {
                    double T_final;
                    int64_t n = og_walk(c, g, xx, yy, ent, NULL, NULL, &T_final, NULL, NULL);
                    int64_t pix = (int64_t)v * HW + (int64_t)yy * c->W + xx;
                    double gC[3], gD = g_depth ? g_depth[pix] : 0.0, gA = g_alpha ? g_alpha[pix] : 0.0;
                    for (int ch = 0; ch < 3; ++ch) gC[ch] = g_rgb ? g_rgb[((int64_t)v * 3 + ch) * HW + (pix - (int64_t)v * HW)] : 0.0;
                    double SC[3], SD = 0.0;
                    for (int ch = 0; ch < 3; ++ch) SC[ch] = T_final * (double)P->bg[ch];
                    for (int64_t k = n - 1; k >= 0; --k) {
                        const og_entry *E = &ent[k];
                        uint32_t f = E->f;
                        int vv = og_view_of(c, f);
                        int64_t gi = P->view_begin[vv] + (f - c->voff[vv]);
                        const double *col = P->c_d + 3 * gi;
                        double a = E->alpha, Tj = E->T, w = a * Tj;
                        double *o = acc + 10 * (int64_t)f;
                        for (int ch = 0; ch < 3; ++ch) OG_ACC(o[7 + ch], gC[ch] * w);
                        OG_ACC(o[6], gD * w);
                        double dLda = gA * T_final / (1.0 - a);
                        for (int ch = 0; ch < 3; ++ch) dLda += gC[ch] * (col[ch] * Tj - SC[ch] / (1.0 - a));
                        dLda += gD * (c->zd[f] * Tj - SD / (1.0 - a));
                        for (int ch = 0; ch < 3; ++ch) SC[ch] += col[ch] * w;
                        SD += c->zd[f] * w;
                        if (E->capped) continue;          /* alpha = alpha_max: no dependence */
                        OG_ACC(o[5], dLda * E->G);              /* d alpha / d o = exp(-sigma) */
                        double dLds = -dLda * a;          /* d alpha / d sigma = -alpha */
                        double dx = E->dx, dy = E->dy;
                        double A = c->cAd[f], B = c->cBd[f], C = c->cCd[f];
                        OG_ACC(o[2], dLds * 0.5 * dx * dx);
                        OG_ACC(o[3], dLds * dx * dy);
                        OG_ACC(o[4], dLds * 0.5 * dy * dy);
                        OG_ACC(o[0], dLds * (-(A * dx + B * dy)));   /* dx = px - mean_x */
                        OG_ACC(o[1], dLds * (-(B * dx + C * dy)));
                    }
                }
        }
        free(ent);
    }
    memset(g2d, 0, sizeof(double) * 10 * c->VN);
    for (int t = 0; t < (shared_acc ? 1 : nthreads); ++t) {
        const double *src = buf + (size_t)t * c->VN * 10;
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < c->VN * 10; ++k) g2d[k] += src[k];
    }
    free(buf);
}

/* ------------------------------------------------------------------------------------------ */
/* 5. projection backward (FP64) and pose gradient                                             */
/*                                                                                              */
/* Pose: left perturbation T <- Exp(xi) T of the world-to-camera pose, xi = (rho, phi), taken   */
/* at xi = 0: d p_c = rho + phi x p_c and d R = [phi]x R.  dL/drho = dL/dp_c and                 */
/* dL/dphi = p_c x dL/dp_c + vee(N - N^T) with N = (dL/dR) R^T.                                   */
/* ------------------------------------------------------------------------------------------ */
static void og_proj_backward_one(const og_ctx *c, int v, int64_t gi, int64_t f, const double *g,
                                 double *g_mu, double *g_ls, double *g_q, double *pose6)
{
    og_p64 o;
    og_project_f64(c, v, gi, f, &o);
    const double *cm = camd(c, v);
    const double *R = cm;
    const double fx = cm[12], fy = cm[13];
    double gmx = g[0], gmy = g[1], gA = g[2], gB = g[3], gC = g[4], gz = g[6];
    double zc = o.pc[2], xc = o.pc[0], yc = o.pc[1];
    double gpc[3] = {0, 0, 0};
    /* mean2D = (fx x/z + cx, fy y/z + cy) */
    gpc[0] += gmx * fx / zc;
    gpc[1] += gmy * fy / zc;
    gpc[2] += -gmx * fx * xc / (zc * zc) - gmy * fy * yc / (zc * zc);
    gpc[2] += gz;                                   /* depth output is z_c */
    /* conic = inverse of [[a, b], [b, c]] */
    double det = o.det, a = o.a, b = o.b, cc = o.c, d2 = det * det;
    double ga = gA * (-cc * cc / d2) + gB * (b * cc / d2) + gC * (1.0 / det - a * cc / d2);
    double gb = gA * (2.0 * b * cc / d2) + gB * (-1.0 / det - 2.0 * b * b / d2) + gC * (2.0 * a * b / d2);
    double gc = gA * (1.0 / det - a * cc / d2) + gB * (a * b / d2) + gC * (-a * a / d2);
    /* a = |U0|^2 + dil, b = U0.U1, c = |U1|^2 + dil */
    double gU[6];
    for (int k = 0; k < 3; ++k) {
        gU[k] = 2.0 * ga * o.U[k] + gb * o.U[3 + k];
        gU[3 + k] = 2.0 * gc * o.U[3 + k] + gb * o.U[k];
    }
    /* U = Wm M */
    double gW[6] = {0}, gM[9] = {0};
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < 3; ++j) {
                gW[3 * r + j] += gU[3 * r + k] * o.M[3 * j + k];
                gM[3 * j + k] += o.Wm[3 * r + j] * gU[3 * r + k];
            }
    /* M = Rq diag(s), s = exp(l) */
    double gRq[9], gs[3] = {0, 0, 0};
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
            gRq[3 * j + k] = gM[3 * j + k] * o.s[k];
            gs[k] += gM[3 * j + k] * o.Rq[3 * j + k];
        }
    for (int k = 0; k < 3; ++k) g_ls[k] += gs[k] * o.s[k];
    /* Rq(q_hat) */
    double w = o.q[0], x = o.q[1], y = o.q[2], z = o.q[3];
    double gqh[4];
    gqh[0] = 2.0 * (-z * gRq[1] + y * gRq[2] + z * gRq[3] - x * gRq[5] - y * gRq[6] + x * gRq[7]);
    gqh[1] = 2.0 * (y * gRq[1] + z * gRq[2] + y * gRq[3] - w * gRq[5] + z * gRq[6] + w * gRq[7])
             - 4.0 * x * (gRq[4] + gRq[8]);
    gqh[2] = 2.0 * (x * gRq[1] + w * gRq[2] + x * gRq[3] + z * gRq[5] - w * gRq[6] + z * gRq[7])
             - 4.0 * y * (gRq[0] + gRq[8]);
    gqh[3] = 2.0 * (-w * gRq[1] + x * gRq[2] + w * gRq[3] + y * gRq[5] + x * gRq[6] + y * gRq[7])
             - 4.0 * z * (gRq[0] + gRq[4]);
    double dotq = gqh[0] * w + gqh[1] * x + gqh[2] * y + gqh[3] * z;
    for (int k = 0; k < 4; ++k) g_q[k] += (gqh[k] - o.q[k] * dotq) / o.qn;
    /* Wm = J R_cam */
    double gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0, gR[9] = {0};
    for (int k = 0; k < 3; ++k) {
        gJ00 += gW[k] * R[k];
        gJ02 += gW[k] * R[6 + k];
        gJ11 += gW[3 + k] * R[3 + k];
        gJ12 += gW[3 + k] * R[6 + k];
        gR[k] += gW[k] * o.J00;
        gR[6 + k] += gW[k] * o.J02 + gW[3 + k] * o.J12;
        gR[3 + k] += gW[3 + k] * o.J11;
    }
    /* J00 = fx/z, J02 = -fx tx / z, tx = x/z unless clamped (then constant) */
    gpc[2] += gJ00 * (-fx / (zc * zc)) + gJ11 * (-fy / (zc * zc));
    gpc[2] += gJ02 * (fx * o.tx / (zc * zc)) + gJ12 * (fy * o.ty / (zc * zc));
    double gtx = gJ02 * (-fx / zc), gty = gJ12 * (-fy / zc);
    if (c->clx[f] == 0) { gpc[0] += gtx / zc; gpc[2] += gtx * (-xc / (zc * zc)); }
    if (c->cly[f] == 0) { gpc[1] += gty / zc; gpc[2] += gty * (-yc / (zc * zc)); }
    /* p_c = R mu + t */
    for (int k = 0; k < 3; ++k) g_mu[k] += R[k] * gpc[0] + R[3 + k] * gpc[1] + R[6 + k] * gpc[2];
    /* pose twist */
    pose6[0] += gpc[0]; pose6[1] += gpc[1]; pose6[2] += gpc[2];
    pose6[3] += yc * gpc[2] - zc * gpc[1];
    pose6[4] += zc * gpc[0] - xc * gpc[2];
    pose6[5] += xc * gpc[1] - yc * gpc[0];
    double N[9] = {0};
    for (int j = 0; j < 3; ++j)
        for (int m = 0; m < 3; ++m)
            for (int k = 0; k < 3; ++k) N[3 * j + m] += gR[3 * j + k] * R[3 * m + k];
    pose6[3] += N[7] - N[5];
    pose6[4] += N[2] - N[6];
    pose6[5] += N[3] - N[1];
}

/* Full backward.  Inputs: dL/drgb [V,3,H,W], dL/ddepth [V,H,W], dL/dalpha [V,H,W] (any may be
 * NULL = 0).  Outputs (all overwritten): g2d [VN,10] (may be NULL), and per Gaussian row
 * g_mu [n,3], g_ls [n,3], g_q [n,4], g_o [n], g_c [n,3] summed over the views that render the row,
 * and g_pose [V,6] ordered (rho_x, rho_y, rho_z, phi_x, phi_y, phi_z). */
void og_backward(const og_ctx *c, const double *g_rgb, const double *g_depth, const double *g_alpha,
                 double *g2d_out, double *g_mu, double *g_ls, double *g_q, double *g_o, double *g_c, double *g_pose)
{
    const og_problem *P = &c->p;
    double *g2d = g2d_out ? g2d_out : (double *)malloc(sizeof(double) * 10 * (c->VN > 0 ? c->VN : 1));
    og_backward_2d(c, g_rgb, g_depth, g_alpha, g2d);
    int64_t n = P->n_gauss;
    memset(g_mu, 0, 24 * n); memset(g_ls, 0, 24 * n); memset(g_q, 0, 32 * n);
    memset(g_o, 0, 8 * n); memset(g_c, 0, 24 * n); memset(g_pose, 0, 48 * c->V);
    for (int v = 0; v < c->V; ++v) {
        int64_t b = P->view_begin[v], nv = P->view_end[v] - b;
        double ps[6] = {0, 0, 0, 0, 0, 0};
#pragma omp parallel
        {
            double pl[6] = {0, 0, 0, 0, 0, 0};
#pragma omp for schedule(static)
            for (int64_t i = 0; i < nv; ++i) {
                int64_t f = c->voff[v] + i, gi = b + i;
                if (!c->touched[f]) continue;
                const double *g = g2d + 10 * f;
                g_o[gi] += g[5];
                for (int ch = 0; ch < 3; ++ch) g_c[3 * gi + ch] += g[7 + ch];
                og_proj_backward_one(c, v, gi, f, g, g_mu + 3 * gi, g_ls + 3 * gi, g_q + 4 * gi, pl);
            }
#pragma omp critical
            for (int k = 0; k < 6; ++k) ps[k] += pl[k];
        }
        for (int k = 0; k < 6; ++k) g_pose[6 * v + k] = ps[k];
    }
    if (!g2d_out) free(g2d);
}
