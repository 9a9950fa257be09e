/*
 * CPU oracle for the differentiable Monte Carlo ray tracer with edge sampling
 * (Karvounas et al. 2021, Section 3.1 "Rendering"; the renderer follows Li et al.
 * 2018, "Differentiable Monte Carlo Ray Tracing through Edge Sampling").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code; only
 * the tests, the smoke check and the bench's CPU-baseline leg load it.
 *
 * Plain and slow on purpose: every ray is tested against every triangle (no
 * acceleration structure), one pixel at a time.  It shares no code with the CUDA
 * library.
 *
 * Precision.  Every quantity that decides an integer or a branch -- the sample
 * jitter, the primary-ray direction, the Moller-Trumbore hit test and closest-hit
 * choice, the vertex normals and the lit/unlit test, the silhouette test, the
 * edge-sample point and its two offset rays, the pixel a point falls in -- is
 * computed in float32 with an explicitly fixed operation order (fmaf where a fused
 * multiply-add is meant, separate * and + otherwise; compiled with
 * -ffp-contract=off).  All values derived from those decisions (shading, pixel
 * means, derivatives, accumulations) are computed in double.
 *
 * Sample streams: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written here from its published definition.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------ */
/* Philox4x32-10                                                                   */
/* ------------------------------------------------------------------------------ */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static float u24(uint32_t r) { return (float)(r >> 8) * 5.9604644775390625e-08f; }

/* ------------------------------------------------------------------------------ */
/* float32 decision arithmetic                                                     */
/* ------------------------------------------------------------------------------ */

typedef struct { float x, y, z; } f3;

static f3 f3_load(const float* p) { f3 r = {p[0], p[1], p[2]}; return r; }
static f3 f3_sub(f3 a, f3 b) { f3 r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static f3 f3_cross(f3 a, f3 b) {
    f3 r = {fmaf(a.y, b.z, -(a.z * b.y)), fmaf(a.z, b.x, -(a.x * b.z)), fmaf(a.x, b.y, -(a.y * b.x))};
    return r;
}
static float f3_dot(f3 a, f3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }

/* camera record: fx fy cx cy R[9] (row-major, world->camera) t[3] centre[3] pad */
typedef struct { float fx, fy, cx, cy, R[9], t[3], c[3], pad; } cam_t;

static void primary_dir(const cam_t* cam, float sx, float sy, f3* d) {
    float dcx = (sx - cam->cx) / cam->fx;
    float dcy = (sy - cam->cy) / cam->fy;
    d->x = fmaf(cam->R[0], dcx, fmaf(cam->R[3], dcy, cam->R[6]));
    d->y = fmaf(cam->R[1], dcx, fmaf(cam->R[4], dcy, cam->R[7]));
    d->z = fmaf(cam->R[2], dcx, fmaf(cam->R[5], dcy, cam->R[8]));
}

typedef struct { int tri; float t, u, v; } hit_t;

/* Moller-Trumbore, double-sided.  Returns 1 and fills t,u,v on a hit. */
static int mt_hit(f3 o, f3 d, f3 v0, f3 e1, f3 e2, float* t_out, float* u_out, float* v_out) {
    f3 p = f3_cross(d, e2);
    float det = f3_dot(e1, p);
    if (det == 0.0f) return 0;
    float inv = 1.0f / det;
    f3 s = f3_sub(o, v0);
    float u = f3_dot(s, p) * inv;
    f3 q = f3_cross(s, e1);
    float v = f3_dot(d, q) * inv;
    float t = f3_dot(e2, q) * inv;
    if (u >= 0.0f && u <= 1.0f && v >= 0.0f && u + v <= 1.0f && t > 0.0f) {
        *t_out = t; *u_out = u; *v_out = v;
        return 1;
    }
    return 0;
}

/* brute force closest hit over all triangles; ties in t go to the lower id */
static hit_t closest_hit(f3 o, f3 d, const float* verts, const int32_t* faces, int F) {
    hit_t h = {-1, INFINITY, 0.0f, 0.0f};
    for (int f = 0; f < F; ++f) {
        f3 v0 = f3_load(verts + 3 * faces[3 * f + 0]);
        f3 v1 = f3_load(verts + 3 * faces[3 * f + 1]);
        f3 v2 = f3_load(verts + 3 * faces[3 * f + 2]);
        f3 e1 = f3_sub(v1, v0), e2 = f3_sub(v2, v0);
        float t, u, v;
        if (mt_hit(o, d, v0, e1, e2, &t, &u, &v)) {
            if (t < h.t) { h.tri = f; h.t = t; h.u = u; h.v = v; }
            /* equal t: the lower id was visited first and is kept */
        }
    }
    return h;
}

void oracle_closest_hits(const float* origins, const float* dirs, int n, const float* verts,
                         const int32_t* faces, int F, int32_t* tri, float* tuv) {
    for (int i = 0; i < n; ++i) {
        hit_t h = closest_hit(f3_load(origins + 3 * i), f3_load(dirs + 3 * i), verts, faces, F);
        tri[i] = h.tri;
        tuv[3 * i] = h.t; tuv[3 * i + 1] = h.u; tuv[3 * i + 2] = h.v;
    }
}

/* area-weighted vertex normals: sum of face cross products over the incident faces
 * in ascending face order, then normalised (zero stays zero) */
void oracle_vertex_normals(const float* verts, int V, const int32_t* faces, const int32_t* vf_off,
                           const int32_t* vf_faces, float* normals) {
    for (int v = 0; v < V; ++v) {
        f3 m = {0.0f, 0.0f, 0.0f};
        for (int k = vf_off[v]; k < vf_off[v + 1]; ++k) {
            int f = vf_faces[k];
            f3 a = f3_load(verts + 3 * faces[3 * f]), b = f3_load(verts + 3 * faces[3 * f + 1]),
               c = f3_load(verts + 3 * faces[3 * f + 2]);
            f3 cf = f3_cross(f3_sub(b, a), f3_sub(c, a));
            m.x = m.x + cf.x; m.y = m.y + cf.y; m.z = m.z + cf.z;
        }
        float len = sqrtf(f3_dot(m, m));
        if (len > 0.0f) { m.x = m.x / len; m.y = m.y / len; m.z = m.z / len; }
        else { m.x = m.y = m.z = 0.0f; }
        normals[3 * v] = m.x; normals[3 * v + 1] = m.y; normals[3 * v + 2] = m.z;
    }
}

/* silhouette edges of one view, ascending edge id; returns the count */
int oracle_silhouettes(const float* verts, const int32_t* faces, const int32_t* edges,
                       const int32_t* edge_faces, int E, const float* cam_rec, int32_t* out) {
    const cam_t* cam = (const cam_t*)cam_rec;
    f3 c = {cam->c[0], cam->c[1], cam->c[2]};
    int n = 0;
    for (int e = 0; e < E; ++e) {
        int f1 = edge_faces[2 * e], f2 = edge_faces[2 * e + 1];
        int sil;
        if (f2 < 0) {
            sil = 1;
        } else {
            f3 w = f3_sub(f3_load(verts + 3 * edges[2 * e]), c);
            int s[2];
            int fs[2] = {f1, f2};
            for (int k = 0; k < 2; ++k) {
                int f = fs[k];
                f3 a = f3_load(verts + 3 * faces[3 * f]), b = f3_load(verts + 3 * faces[3 * f + 1]),
                   cc = f3_load(verts + 3 * faces[3 * f + 2]);
                f3 cf = f3_cross(f3_sub(b, a), f3_sub(cc, a));
                s[k] = f3_dot(cf, w) < 0.0f;
            }
            sil = s[0] != s[1];
        }
        if (sil) out[n++] = e;
    }
    return n;
}

/* ------------------------------------------------------------------------------ */
/* scene and shading                                                               */
/* ------------------------------------------------------------------------------ */

typedef struct {
    uint32_t seed_lo, seed_hi, iter, instance;
    int32_t spp, edge_samples;
    float ka, kd, light_dir[3], light_rgb[3], edge_eps;
    const float* texture;     /* [tex_h][tex_w][3] albedo texture, or NULL: per-vertex albedo */
    const float* uv;          /* [V][2] texture coordinates */
    int32_t tex_w, tex_h;
} opts_t;

/* Bilinear albedo texture at the hit's interpolated uv: texel (i, j) is centred at
 * ((i + 0.5) / W, (j + 0.5) / H), addressing clamps to the edge.  The interpolated uv
 * and the texel coordinates x = uv_x W - 0.5, y = uv_y H - 0.5 (whose floors pick the
 * texels) are float32 decisions; the weights are the fractional parts. */
typedef struct { int i0, i1, j0, j1; double fx, fy; } texs_t;

static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

static texs_t tex_coords(const opts_t* o, const int32_t* f, float u, float v) {
    float w = (1.0f - u) - v;
    const float *t0 = o->uv + 2 * f[0], *t1 = o->uv + 2 * f[1], *t2 = o->uv + 2 * f[2];
    float ux = fmaf(v, t2[0], fmaf(u, t1[0], w * t0[0]));
    float uy = fmaf(v, t2[1], fmaf(u, t1[1], w * t0[1]));
    float x = fmaf(ux, (float)o->tex_w, -0.5f), y = fmaf(uy, (float)o->tex_h, -0.5f);
    float xf = floorf(x), yf = floorf(y);
    texs_t ts;
    ts.fx = (double)(x - xf);
    ts.fy = (double)(y - yf);
    int xi = (int)fminf(fmaxf(xf, -1.0f), (float)o->tex_w), yi = (int)fminf(fmaxf(yf, -1.0f), (float)o->tex_h);
    ts.i0 = clampi(xi, 0, o->tex_w - 1);
    ts.i1 = clampi(xi + 1, 0, o->tex_w - 1);
    ts.j0 = clampi(yi, 0, o->tex_h - 1);
    ts.j1 = clampi(yi + 1, 0, o->tex_h - 1);
    return ts;
}

static double texel(const opts_t* o, int i, int j, int c) { return o->texture[((size_t)j * o->tex_w + i) * 3 + c]; }

static double tex_albedo(const opts_t* o, const texs_t* ts, int c) {
    return (1.0 - ts->fy) * ((1.0 - ts->fx) * texel(o, ts->i0, ts->j0, c) + ts->fx * texel(o, ts->i1, ts->j0, c)) +
           ts->fy * ((1.0 - ts->fx) * texel(o, ts->i0, ts->j1, c) + ts->fx * texel(o, ts->i1, ts->j1, c));
}

typedef struct {
    const float* verts; int V;
    const int32_t* faces; int F;
    const float* normals;     /* float32 vertex normals (decision operand) */
    const float* albedo;
    const cam_t* cams; int N, H, W;
    const float* background;  /* [N][H][W][3] */
    const opts_t* o;
} scene_t;

/* shade a hit: colour in double, computed from the float32 decision operands */
static void shade(const scene_t* sc, const hit_t* h, double rgb[3]) {
    const int32_t* f = sc->faces + 3 * h->tri;
    const float *n0 = sc->normals + 3 * f[0], *n1 = sc->normals + 3 * f[1], *n2 = sc->normals + 3 * f[2];
    const float *a0 = sc->albedo + 3 * f[0], *a1 = sc->albedo + 3 * f[1], *a2 = sc->albedo + 3 * f[2];
    /* lit / unlit decision in float32 */
    float w32 = (1.0f - h->u) - h->v;
    f3 nm32 = {fmaf(h->v, n2[0], fmaf(h->u, n1[0], w32 * n0[0])),
               fmaf(h->v, n2[1], fmaf(h->u, n1[1], w32 * n0[1])),
               fmaf(h->v, n2[2], fmaf(h->u, n1[2], w32 * n0[2]))};
    f3 l32 = {sc->o->light_dir[0], sc->o->light_dir[1], sc->o->light_dir[2]};
    int lit = f3_dot(nm32, l32) > 0.0f;
    double u = h->u, v = h->v, w = 1.0 - u - v;
    double sigma = 0.0;
    if (lit) {
        double nm[3], len2 = 0.0, ndl = 0.0;
        for (int c = 0; c < 3; ++c) {
            nm[c] = w * n0[c] + u * n1[c] + v * n2[c];
            len2 += nm[c] * nm[c];
            ndl += nm[c] * (double)sc->o->light_dir[c];
        }
        sigma = ndl / sqrt(len2);
    }
    texs_t ts;
    if (sc->o->texture) ts = tex_coords(sc->o, f, h->u, h->v);
    for (int c = 0; c < 3; ++c) {
        double alb = sc->o->texture ? tex_albedo(sc->o, &ts, c) : w * a0[c] + u * a1[c] + v * a2[c];
        rgb[c] = alb * (double)sc->o->light_rgb[c] * ((double)sc->o->ka + (double)sc->o->kd * sigma);
    }
}

/* radiance along the ray through screen point (sx, sy) of view `view`; a miss
 * returns background pixel (bpx, bpy) */
static hit_t radiance(const scene_t* sc, int view, float sx, float sy, int bpx, int bpy, double rgb[3]) {
    const cam_t* cam = sc->cams + view;
    f3 d;
    primary_dir(cam, sx, sy, &d);
    f3 o = {cam->c[0], cam->c[1], cam->c[2]};
    hit_t h = closest_hit(o, d, sc->verts, sc->faces, sc->F);
    if (h.tri >= 0) {
        shade(sc, &h, rgb);
    } else {
        const float* b = sc->background + (((size_t)view * sc->H + bpy) * sc->W + bpx) * 3;
        rgb[0] = b[0]; rgb[1] = b[1]; rgb[2] = b[2];
    }
    return h;
}

static void jitter(const scene_t* sc, int view, int px, int py, int s, float* u1, float* u2) {
    uint32_t ctr[4] = {(uint32_t)(py * sc->W + px), (uint32_t)view | (sc->o->instance << 16), (uint32_t)s,
                       (sc->o->iter << 4) | 0u};
    uint32_t key[2] = {sc->o->seed_lo, sc->o->seed_hi};
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    *u1 = u24(r[0]);
    *u2 = u24(r[1]);
}

/* ------------------------------------------------------------------------------ */
/* interior derivative of one shaded hit                                           */
/* ------------------------------------------------------------------------------ */

static void cross_d(const double a[3], const double b[3], double r[3]) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot_d(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* For a hit of the ray (o, d) and upstream weights g[3] = dL/df, add dL/dverts of
 * the triangle (through the barycentrics at the fixed ray) to dV and dL/dnormals
 * to dN.  Barycentrics of the hit: (1-u-v) v0 + u v1 + v v2 = o + t d, with
 * e1 = v1 - v0, e2 = v2 - v0 and [a,b,c] = a.(b x c). */
static void interior_grad(const scene_t* sc, const hit_t* h, f3 o32, f3 d32, const double g[3],
                          double* dV, double* dN, double* dT) {
    const int32_t* f = sc->faces + 3 * h->tri;
    const float* P[3] = {sc->verts + 3 * f[0], sc->verts + 3 * f[1], sc->verts + 3 * f[2]};
    const float *n0 = sc->normals + 3 * f[0], *n1 = sc->normals + 3 * f[1], *n2 = sc->normals + 3 * f[2];
    const float *a0 = sc->albedo + 3 * f[0], *a1 = sc->albedo + 3 * f[1], *a2 = sc->albedo + 3 * f[2];
    const opts_t* op = sc->o;
    double u = h->u, v = h->v, w = 1.0 - u - v;

    float w32 = (1.0f - h->u) - h->v;
    f3 nm32 = {fmaf(h->v, n2[0], fmaf(h->u, n1[0], w32 * n0[0])),
               fmaf(h->v, n2[1], fmaf(h->u, n1[1], w32 * n0[1])),
               fmaf(h->v, n2[2], fmaf(h->u, n1[2], w32 * n0[2]))};
    f3 l32 = {op->light_dir[0], op->light_dir[1], op->light_dir[2]};
    int lit = f3_dot(nm32, l32) > 0.0f;

    double nm[3], len2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        nm[c] = w * n0[c] + u * n1[c] + v * n2[c];
        len2 += nm[c] * nm[c];
    }
    double len = sqrt(len2), nh[3], ndl = 0.0;
    for (int c = 0; c < 3; ++c) { nh[c] = nm[c] / len; ndl += nh[c] * op->light_dir[c]; }
    double sigma = lit ? ndl : 0.0;

    /* dL/dalbedo (per channel) and dL/dsigma */
    texs_t ts;
    if (op->texture) ts = tex_coords(op, f, h->u, h->v);
    double dalb[3], dsig = 0.0;
    for (int c = 0; c < 3; ++c) {
        double alb = op->texture ? tex_albedo(op, &ts, c) : w * a0[c] + u * a1[c] + v * a2[c];
        dalb[c] = g[c] * op->light_rgb[c] * (op->ka + op->kd * sigma);
        dsig += g[c] * alb * op->light_rgb[c] * op->kd;
    }
    /* dL/dnm (unnormalised interpolated normal) */
    double dnm[3] = {0.0, 0.0, 0.0};
    if (lit) {
        double dnh[3] = {dsig * op->light_dir[0], dsig * op->light_dir[1], dsig * op->light_dir[2]};
        double proj = dot_d(nh, dnh);
        for (int c = 0; c < 3; ++c) dnm[c] = (dnh[c] - nh[c] * proj) / len;
    }
    double gu = 0.0, gv = 0.0;
    if (op->texture) {
        /* albedo = bilinear(T, uv(u, v)): dL/dT at the four texels, and dL/duv through
         * the texel coordinates (x = uv_x W - 0.5) to (u, v) */
        double wt[4] = {(1.0 - ts.fx) * (1.0 - ts.fy), ts.fx * (1.0 - ts.fy), (1.0 - ts.fx) * ts.fy, ts.fx * ts.fy};
        int ii[4] = {ts.i0, ts.i1, ts.i0, ts.i1}, jj[4] = {ts.j0, ts.j0, ts.j1, ts.j1};
        double dax = 0.0, day = 0.0;
        for (int c = 0; c < 3; ++c) {
            for (int q = 0; q < 4; ++q) if (dT) dT[((size_t)jj[q] * op->tex_w + ii[q]) * 3 + c] += wt[q] * dalb[c];
            dax += dalb[c] * ((1.0 - ts.fy) * (texel(op, ts.i1, ts.j0, c) - texel(op, ts.i0, ts.j0, c)) +
                              ts.fy * (texel(op, ts.i1, ts.j1, c) - texel(op, ts.i0, ts.j1, c)));
            day += dalb[c] * ((1.0 - ts.fx) * (texel(op, ts.i0, ts.j1, c) - texel(op, ts.i0, ts.j0, c)) +
                              ts.fx * (texel(op, ts.i1, ts.j1, c) - texel(op, ts.i1, ts.j0, c)));
        }
        double dux = dax * op->tex_w, duy = day * op->tex_h;
        const float *q0 = op->uv + 2 * f[0], *q1 = op->uv + 2 * f[1], *q2 = op->uv + 2 * f[2];
        gu += dux * ((double)q1[0] - q0[0]) + duy * ((double)q1[1] - q0[1]);
        gv += dux * ((double)q2[0] - q0[0]) + duy * ((double)q2[1] - q0[1]);
    }
    for (int c = 0; c < 3; ++c) {
        if (!op->texture) {
            gu += dalb[c] * ((double)a1[c] - a0[c]);
            gv += dalb[c] * ((double)a2[c] - a0[c]);
        }
        gu += dnm[c] * ((double)n1[c] - n0[c]);
        gv += dnm[c] * ((double)n2[c] - n0[c]);
        dN[3 * f[0] + c] += w * dnm[c];
        dN[3 * f[1] + c] += u * dnm[c];
        dN[3 * f[2] + c] += v * dnm[c];
    }
    /* barycentric derivatives at the fixed ray: the hit solves
     * (1-u-v) v0 + u v1 + v v2 = o + t d, so moving vertex k by dp changes (u, v, t)
     * by -M^-1 (w_k dp) with M = [e1, e2, -d] and w = (1-u-v, u, v).  Rows 0 and 1 of
     * M^-1 are (d x e2) / D and (e1 x d) / D with D = e1 . (d x e2), hence
     *   dL/dv_k = -w_k (gu (d x e2) + gv (e1 x d)) / D.
     * (The equivalent form through s = o - v0 holds only when (u, v) solve the
     * system exactly; with the float32 hit's (u, v) it loses ~|s| / |e| of their
     * precision, while this one depends on them linearly.) */
    double dd[3] = {d32.x, d32.y, d32.z};
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = (double)P[1][c] - P[0][c];
        e2[c] = (double)P[2][c] - P[0][c];
    }
    (void)o32;
    double dxe2[3], e1xd[3];
    cross_d(dd, e2, dxe2);        /* d x e2 */
    cross_d(e1, dd, e1xd);        /* e1 x d */
    double D = dot_d(e1, dxe2);   /* [e1, d, e2] */
    for (int c = 0; c < 3; ++c) {
        double q = (gu * dxe2[c] + gv * e1xd[c]) / D;
        dV[3 * f[0] + c] -= w * q;
        dV[3 * f[1] + c] -= u * q;
        dV[3 * f[2] + c] -= v * q;
    }
}

/* ------------------------------------------------------------------------------ */
/* threaded drivers                                                                */
/* ------------------------------------------------------------------------------ */

typedef struct {
    const scene_t* sc;
    int item0, item1;          /* rows [item0, item1) over N*H */
    double* image;             /* forward output [N][H][W][3] (NULL in backward) */
    const float* adjoint;      /* backward input [N][H][W][3] */
    double* dV; double* dN;    /* private accumulators [V][3] */
    double* dT;                /* private texture accumulator [tex_h][tex_w][3] or NULL */
    int col0, col1;            /* column range */
} job_t;

static void* fwd_worker(void* arg) {
    job_t* j = (job_t*)arg;
    const scene_t* sc = j->sc;
    for (int item = j->item0; item < j->item1; ++item) {
        int view = item / sc->H, py = item % sc->H;
        for (int px = j->col0; px < j->col1; ++px) {
            double acc[3] = {0.0, 0.0, 0.0};
            for (int s = 0; s < sc->o->spp; ++s) {
                float u1, u2;
                jitter(sc, view, px, py, s, &u1, &u2);
                double rgb[3];
                /* a primary sample estimates pixel (px, py): its miss value is that
                 * pixel's background even when px + u1 rounds up to px + 1 */
                radiance(sc, view, (float)px + u1, (float)py + u2, px, py, rgb);
                acc[0] += rgb[0]; acc[1] += rgb[1]; acc[2] += rgb[2];
            }
            double* out = j->image + (((size_t)view * sc->H + py) * sc->W + px) * 3;
            for (int c = 0; c < 3; ++c) out[c] = acc[c] / sc->o->spp;
        }
    }
    return NULL;
}

static void* bwd_worker(void* arg) {
    job_t* j = (job_t*)arg;
    const scene_t* sc = j->sc;
    for (int item = j->item0; item < j->item1; ++item) {
        int view = item / sc->H, py = item % sc->H;
        const cam_t* cam = sc->cams + view;
        f3 o = {cam->c[0], cam->c[1], cam->c[2]};
        for (int px = j->col0; px < j->col1; ++px) {
            const float* A = j->adjoint + (((size_t)view * sc->H + py) * sc->W + px) * 3;
            if (A[0] == 0.0f && A[1] == 0.0f && A[2] == 0.0f) continue;
            double g[3] = {(double)A[0] / sc->o->spp, (double)A[1] / sc->o->spp, (double)A[2] / sc->o->spp};
            for (int s = 0; s < sc->o->spp; ++s) {
                float u1, u2;
                jitter(sc, view, px, py, s, &u1, &u2);
                f3 d;
                primary_dir(cam, (float)px + u1, (float)py + u2, &d);
                hit_t h = closest_hit(o, d, sc->verts, sc->faces, sc->F);
                if (h.tri >= 0) interior_grad(sc, &h, o, d, g, j->dV, j->dN, j->dT);
            }
        }
    }
    return NULL;
}

static void run_jobs(const scene_t* sc, int nthreads, int row0, int row1, int col0, int col1, double* image,
                     const float* adjoint, double* dV, double* dN, double* dT, void* (*fn)(void*)) {
    if (nthreads < 1) nthreads = 1;
    int rows = row1 - row0;
    if (nthreads > rows) nthreads = rows > 0 ? rows : 1;
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    job_t* jobs = (job_t*)calloc((size_t)nthreads, sizeof(job_t));
    size_t nv = (size_t)sc->V * 3;
    size_t nt = dT ? (size_t)sc->o->tex_w * sc->o->tex_h * 3 : 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].sc = sc;
        jobs[t].item0 = row0 + (int)((long)rows * t / nthreads);
        jobs[t].item1 = row0 + (int)((long)rows * (t + 1) / nthreads);
        jobs[t].col0 = col0; jobs[t].col1 = col1;
        jobs[t].image = image;
        jobs[t].adjoint = adjoint;
        if (dV) {
            jobs[t].dV = (double*)calloc(nv, sizeof(double));
            jobs[t].dN = (double*)calloc(nv, sizeof(double));
        }
        if (nt) jobs[t].dT = (double*)calloc(nt, sizeof(double));
        pthread_create(&th[t], NULL, fn, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    if (dV) {
        for (int t = 0; t < nthreads; ++t) {
            for (size_t i = 0; i < nv; ++i) { dV[i] += jobs[t].dV[i]; dN[i] += jobs[t].dN[i]; }
            free(jobs[t].dV); free(jobs[t].dN);
        }
    }
    for (int t = 0; t < nthreads && nt; ++t) {
        for (size_t i = 0; i < nt; ++i) dT[i] += jobs[t].dT[i];
        free(jobs[t].dT);
    }
    free(th); free(jobs);
}

static void make_scene(scene_t* sc, const float* verts, int V, const int32_t* faces, int F, const float* normals,
                       const float* albedo, const float* cams, int N, int H, int W, const float* background,
                       const opts_t* o) {
    sc->verts = verts; sc->V = V; sc->faces = faces; sc->F = F; sc->normals = normals; sc->albedo = albedo;
    sc->cams = (const cam_t*)cams; sc->N = N; sc->H = H; sc->W = W; sc->background = background; sc->o = o;
}

/* Forward render: image[p] = (1/spp) sum_s f(x_s) over rows [row0,row1) of the
 * N*H stacked rows and columns [col0,col1) (the full image is 0,N*H,0,W). */
void oracle_render_fwd(const float* verts, int V, const int32_t* faces, int F, const float* normals,
                       const float* albedo, const float* cams, int N, int H, int W, const float* background,
                       const opts_t* o, double* image, int nthreads, int row0, int row1, int col0, int col1) {
    scene_t sc;
    make_scene(&sc, verts, V, faces, F, normals, albedo, cams, N, H, W, background, o);
    run_jobs(&sc, nthreads, row0, row1, col0, col1, image, NULL, NULL, NULL, NULL, fwd_worker);
}

/* Interior backward: re-trace the forward's samples and accumulate dL/dV (through
 * the barycentrics), dL/dN (vertex normals) and, with a texture, dL/dtexture (dT, or
 * NULL) for adjoint image A = dL/dI. */
void oracle_render_bwd_interior(const float* verts, int V, const int32_t* faces, int F, const float* normals,
                                const float* albedo, const float* cams, int N, int H, int W,
                                const float* background, const opts_t* o, const float* adjoint, double* dV,
                                double* dN, double* dT, int nthreads, int row0, int row1, int col0, int col1) {
    scene_t sc;
    make_scene(&sc, verts, V, faces, F, normals, albedo, cams, N, H, W, background, o);
    run_jobs(&sc, nthreads, row0, row1, col0, col1, NULL, adjoint, dV, dN, o->texture ? dT : NULL, bwd_worker);
}

/* project a vertex; returns 0 when it is not in front of the camera */
static int project32(const cam_t* cam, const float* v, float* ax, float* ay) {
    float X = fmaf(cam->R[0], v[0], fmaf(cam->R[1], v[1], fmaf(cam->R[2], v[2], cam->t[0])));
    float Y = fmaf(cam->R[3], v[0], fmaf(cam->R[4], v[1], fmaf(cam->R[5], v[2], cam->t[1])));
    float Z = fmaf(cam->R[6], v[0], fmaf(cam->R[7], v[1], fmaf(cam->R[8], v[2], cam->t[2])));
    if (!(Z > 1e-3f)) return 0;
    *ax = fmaf(cam->fx, X / Z, cam->cx);
    *ay = fmaf(cam->fy, Y / Z, cam->cy);
    return 1;
}

/* d(screen point)/d(vertex) of the pinhole projection, in double: 2x3 */
static void project_jacobian(const cam_t* cam, const float* v, double J[2][3]) {
    double P[3];
    for (int r = 0; r < 3; ++r)
        P[r] = (double)cam->R[3 * r] * v[0] + (double)cam->R[3 * r + 1] * v[1] + (double)cam->R[3 * r + 2] * v[2] +
               cam->t[r];
    double iz = 1.0 / P[2];
    for (int c = 0; c < 3; ++c) {
        J[0][c] = cam->fx * iz * ((double)cam->R[c] - P[0] * iz * cam->R[6 + c]);
        J[1][c] = cam->fy * iz * ((double)cam->R[3 + c] - P[1] * iz * cam->R[6 + c]);
    }
}

/* Edge-sampling backward for one view (boundary term of the pixel-integral
 * derivative).  Samples: edge uniform over the view's silhouette list, point
 * uniform along it; f+ and f- are traced at the point offset by +-eps along the
 * unit screen normal of alpha (the side where alpha > 0 is "+").  The per-sample
 * contribution to dL/d(endpoint) is A[p(x)].(f+ - f-) * dalpha/d(endpoint) * N_sil,
 * averaged over the view's samples, then mapped to vertices. */
void oracle_render_bwd_edges(const float* verts, int V, const int32_t* faces, int F, const float* normals,
                             const float* albedo, const float* cams, int N, int H, int W, const float* background,
                             const opts_t* o, const float* adjoint, const int32_t* edges, const int32_t* sil,
                             const int32_t* sil_count, int sil_stride, double* dV, int k0, int k1) {
    scene_t sc;
    make_scene(&sc, verts, V, faces, F, normals, albedo, cams, N, H, W, background, o);
    for (int view = 0; view < N; ++view) {
        const cam_t* cam = sc.cams + view;
        int nsil = sil_count[view];
        if (nsil == 0 || o->edge_samples <= 0) continue;
        double scale = (double)nsil / (double)o->edge_samples;
        for (int k = k0; k < k1 && k < o->edge_samples; ++k) {
            uint32_t ctr[4] = {(uint32_t)k, (uint32_t)view | (o->instance << 16), 0u, (o->iter << 4) | 1u};
            uint32_t key[2] = {o->seed_lo, o->seed_hi};
            uint32_t r[4];
            oracle_philox4x32_10(ctr, key, r);
            int si = (int)(((uint64_t)r[0] * (uint64_t)nsil) >> 32);
            float t = u24(r[1]);
            int e = sil[(size_t)view * sil_stride + si];
            int ia = edges[2 * e], ib = edges[2 * e + 1];
            float ax, ay, bx, by;
            if (!project32(cam, verts + 3 * ia, &ax, &ay)) continue;
            if (!project32(cam, verts + 3 * ib, &bx, &by)) continue;
            float x = fmaf(t, bx - ax, ax), y = fmaf(t, by - ay, ay);
            float nx = ay - by, ny = bx - ax;
            float len = sqrtf(fmaf(nx, nx, ny * ny));
            if (!(len > 0.0f)) continue;
            float nhx = nx / len, nhy = ny / len;
            float fx_ = floorf(x), fy_ = floorf(y);
            if (fx_ < 0.0f || fy_ < 0.0f || fx_ >= (float)W || fy_ >= (float)H) continue;
            int px = (int)fx_, py = (int)fy_;
            const float* A = adjoint + (((size_t)view * H + py) * W + px) * 3;
            if (A[0] == 0.0f && A[1] == 0.0f && A[2] == 0.0f) continue;
            float xp = fmaf(o->edge_eps, nhx, x), yp = fmaf(o->edge_eps, nhy, y);
            float xm = fmaf(-o->edge_eps, nhx, x), ym = fmaf(-o->edge_eps, nhy, y);
            /* offset rays that miss see the background pixel containing the
             * offset point, clamped to the image */
            int bxp = (int)fminf(fmaxf(floorf(xp), 0.0f), (float)(W - 1));
            int byp = (int)fminf(fmaxf(floorf(yp), 0.0f), (float)(H - 1));
            int bxm = (int)fminf(fmaxf(floorf(xm), 0.0f), (float)(W - 1));
            int bym = (int)fminf(fmaxf(floorf(ym), 0.0f), (float)(H - 1));
            double fp[3], fm[3];
            radiance(&sc, view, xp, yp, bxp, byp, fp);
            radiance(&sc, view, xm, ym, bxm, bym, fm);
            double wgt = 0.0;
            for (int c = 0; c < 3; ++c) wgt += (double)A[c] * (fp[c] - fm[c]);
            if (wgt == 0.0) continue;
            wgt *= scale;
            double X = x, Y = y;
            double dax = wgt * ((double)by - Y), day = wgt * (X - (double)bx);
            double dbx = wgt * (Y - (double)ay), dby = wgt * ((double)ax - X);
            double Ja[2][3], Jb[2][3];
            project_jacobian(cam, verts + 3 * ia, Ja);
            project_jacobian(cam, verts + 3 * ib, Jb);
            for (int c = 0; c < 3; ++c) {
                dV[3 * ia + c] += dax * Ja[0][c] + day * Ja[1][c];
                dV[3 * ib + c] += dbx * Jb[0][c] + dby * Jb[1][c];
            }
        }
    }
}
