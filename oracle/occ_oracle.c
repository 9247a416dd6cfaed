/*
 * occ_oracle.c -- plain, slow FP64 CPU oracle for occlusion-point reuse.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant generator with the CUDA library; the two meet only in the
 * seeded input data (triangles, G-buffers, cameras, lights, offsets).
 *
 * Everything is computed in double precision from float inputs widened
 * exactly.  There is no blocking, fusion or reordering beyond what the
 * definitions state.  Sections and what they follow:
 *
 *   Philox4x32-10 ........ Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 *                          as easy as 1, 2, 3", SC'11 (counter-based generator).
 *   AO direction ......... Eq. 2: cosine-weighted hemisphere (Malley's method),
 *                          tangent frame from Duff et al., JCGT 2017.
 *   Shadow sample ........ Eq. 5: uniform point on the rectangle light.
 *   Closest hit .......... first intersection along a ray (Eq. 7, Alg. 1/2
 *                          step 1); watertight test of Woop, Benthin, Wald,
 *                          JCGT 2013, evaluated in FP64; a median-split binary
 *                          BVH or brute force over all triangles.
 *   Neighbour sets ....... Eq. 8: group blocks, centred box, shared offsets, and
 *                          per-receiver random offsets in a disk (drawn with Philox).
 *   Densities ............ Eq. 15 (AO) and Eqs. 20-21 (shadow); with the
 *                          first-hit predicate (unbiased) or without it
 *                          (biased, Eqs. 18 and 24).
 *   Estimator ............ Eqs. 17, 18, 23, 24 and Algorithms 1-2 step 3,
 *                          plus the all-blocked guard of Sec. 4.4.
 *   Baselines ............ Eqs. 3 and 6 (no reuse); box mean of visibility.
 *
 * Readings where the paper is silent are listed with the functions below:
 * the receiver point is the G-buffer position (already offset along its
 * normal), the AO radius test is inclusive with a 2^-16 relative slack on R^2,
 * the light is one-sided with its rectangle test inclusive with the same
 * slack, first-hit validation compares triangle ids of the closest hit, and
 * estimates are never clamped.
 *
 * "Margins": every query also returns the smallest normalised distance of any
 * decision it took (inside/outside a triangle edge, t against its interval,
 * support tests of the densities) from its threshold.  A tiny margin marks a
 * result that an FP32 evaluation may legitimately decide the other way.
 *
 * Plain C11; builds with gcc on x86-64 and aarch64 without fast-math and
 * with floating-point contraction off, so both machines round alike.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ----------------------------------------------------------------------------------
 * Philox4x32-10 (SC'11).  One round maps (x0, x1, x2, x3) with key (k0, k1) to
 *   (hi(B*x2) ^ x1 ^ k0,  lo(B*x2),  hi(A*x0) ^ x3 ^ k1,  lo(A*x0))
 * with multipliers A = 0xD2511F53, B = 0xCD9E8D57; the key is bumped by the
 * Weyl constants (0x9E3779B9, 0xBB67AE85) between rounds.  Ten rounds.
 * -------------------------------------------------------------------------------- */
ORC_API void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t n0 = (uint32_t)(pb >> 32) ^ x1 ^ k0;
        uint32_t n1 = (uint32_t)pb;
        uint32_t n2 = (uint32_t)(pa >> 32) ^ x3 ^ k1;
        uint32_t n3 = (uint32_t)pa;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Stream ids of the counter's third word. */
enum { ORC_STREAM_AO = 0, ORC_STREAM_SHADOW = 1 };

/* Two uniforms in [0, 1) for (pixel, sample, stream): the top 24 bits of the
 * first two output words, scaled by 2^-24 (exact in FP32 and FP64). */
static void rng_pair(uint64_t seed, uint32_t pix, uint32_t sample, uint32_t stream,
                     double* u1, double* u2) {
    uint32_t ctr[4] = {pix, sample, stream, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    *u1 = (double)(o[0] >> 8) * (1.0 / 16777216.0);
    *u2 = (double)(o[1] >> 8) * (1.0 / 16777216.0);
}

ORC_API void orc_uniform_pair(uint64_t seed, uint32_t pix, uint32_t sample, uint32_t stream,
                              double out[2]) {
    rng_pair(seed, pix, sample, stream, &out[0], &out[1]);
}

/* ----------------------------------------------------------------------------------
 * Small vector helpers
 * -------------------------------------------------------------------------------- */
typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static v3 normalize(v3 a) { return scl(a, 1.0 / sqrt(dot(a, a))); }
static double comp(v3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }
static v3 ldf(const float* p) { return mk((double)p[0], (double)p[1], (double)p[2]); }

/* ----------------------------------------------------------------------------------
 * Eq. 2: cosine-weighted direction about n.  Malley's method maps (u1, u2) to
 * the unit disk (r = sqrt(u1), phi = 2 pi u2) and lifts it to the hemisphere.
 * The tangent frame (t, b, n) is the branch-free basis of Duff et al. 2017.
 * -------------------------------------------------------------------------------- */
static void onb(v3 n, v3* t, v3* b) {
    double s = copysign(1.0, n.z);
    double a = -1.0 / (s + n.z);
    double c = n.x * n.y * a;
    *t = mk(1.0 + s * n.x * n.x * a, s * c, -s * n.x);
    *b = mk(c, s + n.y * n.y * a, -n.y);
}

static v3 cosine_dir(v3 n, double u1, double u2) {
    double r = sqrt(u1), phi = 2.0 * M_PI * u2;
    double lx = r * cos(phi), ly = r * sin(phi), lz = sqrt(fmax(0.0, 1.0 - u1));
    v3 t, b;
    onb(n, &t, &b);
    return add(add(scl(t, lx), scl(b, ly)), scl(n, lz));
}

/* ----------------------------------------------------------------------------------
 * Rectangle light: c + a eu + b ev, a, b in [-1/2, 1/2].  Emitting normal
 * nL = normalize(eu x ev); Area = |eu x ev| (eu and ev orthogonal).
 * -------------------------------------------------------------------------------- */
typedef struct { v3 c, eu, ev, n; double eu2, ev2, area; } light_t;

static light_t mk_light(const float* L) {
    light_t l;
    l.c = ldf(L); l.eu = ldf(L + 3); l.ev = ldf(L + 6);
    v3 cr = cross(l.eu, l.ev);
    l.area = sqrt(dot(cr, cr));
    l.n = scl(cr, 1.0 / l.area);
    l.eu2 = dot(l.eu, l.eu);
    l.ev2 = dot(l.ev, l.ev);
    return l;
}

/* ----------------------------------------------------------------------------------
 * Scene: triangles widened to double, median-split binary BVH.
 * -------------------------------------------------------------------------------- */
typedef struct {
    int64_t T;
    double* v;          /* T * 9 */
    int64_t n_nodes;
    double* lo;         /* n_nodes * 3 */
    double* hi;
    int64_t* kid;       /* n_nodes * 2: children, or (-1 - first, count) for a leaf */
    int64_t* perm;      /* leaf ranges index this permutation of triangle ids */
    double pad;         /* absolute box padding */
} scene_t;

static double tri_c(const scene_t* s, int64_t t, int axis) {
    const double* v = s->v + 9 * t;
    return (v[axis] + v[3 + axis] + v[6 + axis]) / 3.0;
}

/* Quickselect: place the k-th smallest centroid (along axis) of perm[lo..hi) at k. */
static void select_k(const scene_t* s, int64_t* perm, int64_t lo, int64_t hi, int64_t k, int axis) {
    while (hi - lo > 1) {
        double pivot = tri_c(s, perm[lo + (hi - lo) / 2], axis);
        int64_t i = lo, j = hi - 1;
        while (i <= j) {
            while (tri_c(s, perm[i], axis) < pivot) ++i;
            while (tri_c(s, perm[j], axis) > pivot) --j;
            if (i <= j) { int64_t tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp; ++i; --j; }
        }
        if (k <= j) hi = j + 1;
        else if (k >= i) lo = i;
        else return;
    }
}

typedef struct { int64_t node, first, count; } build_item;

static void build_bvh(scene_t* s) {
    int64_t T = s->T;
    int64_t cap = 2 * T + 1;
    s->lo = (double*)malloc(sizeof(double) * 3 * cap);
    s->hi = (double*)malloc(sizeof(double) * 3 * cap);
    s->kid = (int64_t*)malloc(sizeof(int64_t) * 2 * cap);
    s->perm = (int64_t*)malloc(sizeof(int64_t) * (T > 0 ? T : 1));
    for (int64_t i = 0; i < T; ++i) s->perm[i] = i;
    s->n_nodes = 1;
    build_item* stack = (build_item*)malloc(sizeof(build_item) * 256);
    int sp = 0;
    stack[sp].node = 0; stack[sp].first = 0; stack[sp].count = T; ++sp;
    while (sp > 0) {
        build_item it = stack[--sp];
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = it.first; i < it.first + it.count; ++i) {
            const double* v = s->v + 9 * s->perm[i];
            for (int a = 0; a < 3; ++a) {
                for (int q = 0; q < 3; ++q) {
                    lo[a] = fmin(lo[a], v[3 * q + a]);
                    hi[a] = fmax(hi[a], v[3 * q + a]);
                }
                double c = tri_c(s, s->perm[i], a);
                clo[a] = fmin(clo[a], c);
                chi[a] = fmax(chi[a], c);
            }
        }
        for (int a = 0; a < 3; ++a) {
            double p = 1e-4 * (hi[a] - lo[a]) + s->pad;
            s->lo[3 * it.node + a] = lo[a] - p;
            s->hi[3 * it.node + a] = hi[a] + p;
        }
        if (it.count <= 4) {
            s->kid[2 * it.node] = -1 - it.first;
            s->kid[2 * it.node + 1] = it.count;
            continue;
        }
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
        int64_t half = it.count / 2;
        select_k(s, s->perm, it.first, it.first + it.count, it.first + half, axis);
        int64_t l = s->n_nodes++, r = s->n_nodes++;
        s->kid[2 * it.node] = l;
        s->kid[2 * it.node + 1] = r;
        stack[sp].node = l; stack[sp].first = it.first; stack[sp].count = half; ++sp;
        stack[sp].node = r; stack[sp].first = it.first + half; stack[sp].count = it.count - half; ++sp;
    }
    free(stack);
}

ORC_API void* orc_scene_create(const float* tris, int64_t T) {
    scene_t* s = (scene_t*)calloc(1, sizeof(scene_t));
    s->T = T;
    s->v = (double*)malloc(sizeof(double) * 9 * (T > 0 ? T : 1));
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < 9 * T; ++i) {
        s->v[i] = (double)tris[i];
        lo = fmin(lo, s->v[i]);
        hi = fmax(hi, s->v[i]);
    }
    s->pad = T > 0 ? 1e-6 * (hi - lo) + 1e-9 : 0.0;
    if (T > 0) build_bvh(s);
    return s;
}

ORC_API void orc_scene_destroy(void* p) {
    scene_t* s = (scene_t*)p;
    if (!s) return;
    free(s->v); free(s->lo); free(s->hi); free(s->kid); free(s->perm);
    free(s);
}

ORC_API int64_t orc_scene_nodes(const void* p) { return ((const scene_t*)p)->n_nodes; }

/* ----------------------------------------------------------------------------------
 * Watertight ray/triangle test (Woop, Benthin, Wald 2013) in FP64.
 * The ray is sheared so that it runs along +z; the edge functions U, V, W of
 * the projected triangle decide inside (all of one sign, zeros allowed) and
 * T / det is the hit distance in units of the direction vector.  Two-sided.
 * -------------------------------------------------------------------------------- */
typedef struct { int kx, ky, kz; double Sx, Sy, Sz; v3 o; } wray;

static void wray_init(wray* r, v3 o, v3 d) {
    double a[3] = {fabs(d.x), fabs(d.y), fabs(d.z)};
    int kz = 0;
    if (a[1] > a[kz]) kz = 1;
    if (a[2] > a[kz]) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    double dz = comp(d, kz);
    if (dz < 0.0) { int tmp = kx; kx = ky; ky = tmp; }
    r->kx = kx; r->ky = ky; r->kz = kz;
    r->Sx = comp(d, kx) / dz;
    r->Sy = comp(d, ky) / dz;
    r->Sz = 1.0 / dz;
    r->o = o;
}

/* Returns the plane distance in *tp and the smallest normalised barycentric
 * coordinate in *bmin (>= 0 inside).  Returns 0 for a degenerate projection. */
static int wt_eval(const wray* r, const double* v, double* tp, double* bmin) {
    v3 A = sub(mk(v[0], v[1], v[2]), r->o);
    v3 B = sub(mk(v[3], v[4], v[5]), r->o);
    v3 C = sub(mk(v[6], v[7], v[8]), r->o);
    double Ax = comp(A, r->kx) - r->Sx * comp(A, r->kz);
    double Ay = comp(A, r->ky) - r->Sy * comp(A, r->kz);
    double Bx = comp(B, r->kx) - r->Sx * comp(B, r->kz);
    double By = comp(B, r->ky) - r->Sy * comp(B, r->kz);
    double Cx = comp(C, r->kx) - r->Sx * comp(C, r->kz);
    double Cy = comp(C, r->ky) - r->Sy * comp(C, r->kz);
    double U = Cx * By - Cy * Bx;
    double V = Ax * Cy - Ay * Cx;
    double W = Bx * Ay - By * Ax;
    double det = U + V + W;
    if (det == 0.0) return 0;
    double Az = r->Sz * comp(A, r->kz);
    double Bz = r->Sz * comp(B, r->kz);
    double Cz = r->Sz * comp(C, r->kz);
    double Tn = U * Az + V * Bz + W * Cz;
    *tp = Tn / det;
    *bmin = fmin(U / det, fmin(V / det, W / det));
    return 1;
}

/* ----------------------------------------------------------------------------------
 * Closest hit on the interval (0, tmax]; ties go to the smaller t, then the
 * smaller triangle id.  The margin is the smallest of: the barycentric
 * distance to an edge, |t - tmax| / tmax and t / tmax, and the relative t gap
 * to the best hit, over every triangle that could change the answer (plane
 * distance within (-delta tmax, min(t_best, tmax)(1 + delta)]).
 * -------------------------------------------------------------------------------- */
typedef struct { int64_t tri; double t, margin; } hit_t;

#define MARGIN_DELTA 1e-3

typedef struct { int64_t id; double tp, bmin; } cand_t;

static void consider(const wray* r, const scene_t* s, int64_t id, double tmax, hit_t* best,
                     cand_t* near, int* n_near, int cap) {
    double tp, bmin;
    if (!wt_eval(r, s->v + 9 * id, &tp, &bmin)) return;
    if (!(tp > -MARGIN_DELTA * tmax && tp <= tmax * (1.0 + MARGIN_DELTA))) return;
    if (bmin < -MARGIN_DELTA) return;
    int inside = bmin >= 0.0;
    if (inside && tp > 0.0 && tp <= tmax) {
        if (best->tri < 0 || tp < best->t || (tp == best->t && id < best->tri)) {
            best->tri = id;
            best->t = tp;
        }
    }
    if (*n_near < cap) {
        near[*n_near].id = id; near[*n_near].tp = tp; near[*n_near].bmin = bmin;
        ++*n_near;
    } else {
        best->margin = 0.0;   /* too many near candidates: treat as ambiguous */
    }
}

static double finish_margin(const hit_t* best, const cand_t* near, int n_near, double tmax) {
    double m = best->margin;
    double tcut = (best->tri >= 0 ? best->t : tmax) * (1.0 + MARGIN_DELTA);
    for (int i = 0; i < n_near; ++i) {
        const cand_t* c = &near[i];
        if (c->tp > tcut) continue;
        double range = fmin(fabs(c->tp - tmax) / tmax, fabs(c->tp) / tmax);
        double mi;
        if (best->tri >= 0 && c->id == best->tri) {
            /* the chosen hit: it may slip across an edge or out of the interval */
            mi = fmin(c->bmin, range);
        } else if (c->bmin >= 0.0) {
            /* inside another triangle: it may win on t, or enter the interval */
            int in_range = c->tp > 0.0 && c->tp <= tmax;
            mi = in_range ? (best->tri >= 0 ? fabs(c->tp - best->t) / best->t : 0.0) : range;
        } else {
            /* just outside another triangle closer than the answer: it may turn inside */
            mi = -c->bmin;
        }
        m = fmin(m, mi);
    }
    return m;
}

#define NEAR_CAP 256

static hit_t closest_hit(const scene_t* s, v3 o, v3 d, double tmax, int brute) {
    hit_t best = {-1, tmax, INFINITY};
    cand_t near[NEAR_CAP];
    int n_near = 0;
    if (s->T == 0) return best;
    wray r;
    wray_init(&r, o, d);
    if (brute) {
        for (int64_t i = 0; i < s->T; ++i) consider(&r, s, i, tmax, &best, near, &n_near, NEAR_CAP);
    } else {
        double inv[3] = {1.0 / d.x, 1.0 / d.y, 1.0 / d.z};
        double oo[3] = {o.x, o.y, o.z};
        int64_t stack[256];
        int sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            int64_t nd = stack[--sp];
            double t0 = -MARGIN_DELTA * tmax;
            double t1 = (best.tri >= 0 ? best.t : tmax) * (1.0 + MARGIN_DELTA);
            int ok = 1;
            for (int a = 0; a < 3 && ok; ++a) {
                double lo = s->lo[3 * nd + a], hi = s->hi[3 * nd + a];
                if (inv[a] == INFINITY || inv[a] == -INFINITY) {
                    if (oo[a] < lo || oo[a] > hi) ok = 0;
                    continue;
                }
                double ta = (lo - oo[a]) * inv[a], tb = (hi - oo[a]) * inv[a];
                t0 = fmax(t0, fmin(ta, tb));
                t1 = fmin(t1, fmax(ta, tb));
                if (t0 > t1) ok = 0;
            }
            if (!ok) continue;
            int64_t k0 = s->kid[2 * nd], k1 = s->kid[2 * nd + 1];
            if (k0 < 0) {
                int64_t first = -1 - k0;
                for (int64_t i = first; i < first + k1; ++i)
                    consider(&r, s, s->perm[i], tmax, &best, near, &n_near, NEAR_CAP);
            } else {
                if (sp + 2 > 256) { best.margin = 0.0; continue; }
                stack[sp++] = k1;
                stack[sp++] = k0;
            }
        }
    }
    best.margin = finish_margin(&best, near, n_near, tmax);
    if (best.tri < 0) best.t = tmax;
    return best;
}

ORC_API void orc_closest_hit_batch(const void* sc, int64_t n, const double* o, const double* d,
                                   const double* tmax, int brute, int64_t* tri, double* t,
                                   double* margin) {
    const scene_t* s = (const scene_t*)sc;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        hit_t h = closest_hit(s, mk(o[3 * i], o[3 * i + 1], o[3 * i + 2]),
                              mk(d[3 * i], d[3 * i + 1], d[3 * i + 2]), tmax[i], brute);
        tri[i] = h.tri;
        t[i] = h.t;
        margin[i] = h.margin;
    }
}

/* Geometric unit normal of a triangle (orientation by vertex order). */
static v3 tri_normal(const scene_t* s, int64_t id) {
    const double* v = s->v + 9 * id;
    v3 e1 = sub(mk(v[3], v[4], v[5]), mk(v[0], v[1], v[2]));
    v3 e2 = sub(mk(v[6], v[7], v[8]), mk(v[0], v[1], v[2]));
    return normalize(cross(e1, e2));
}

/* ----------------------------------------------------------------------------------
 * G-buffer producer (input stage, not part of the method): a pinhole camera
 * (eye, target, up, vertical fov in degrees) casts one primary ray through
 * each pixel centre.  The stored position is the receiver point: the hit
 * point pushed eps along the geometric normal turned toward the camera.
 * Output: float pos4 (w = 1 valid, all zero on a miss) and nrm4 (w = 0).
 * -------------------------------------------------------------------------------- */
ORC_API void orc_gbuffer(const void* sc, const float* cam, int W, int H, float eps,
                         float* pos4, float* nrm4, int64_t* tri_out) {
    const scene_t* s = (const scene_t*)sc;
    v3 eye = ldf(cam), tgt = ldf(cam + 3), up = ldf(cam + 6);
    double th = tan(0.5 * (double)cam[9] * M_PI / 180.0);
    double aspect = (double)W / (double)H;
    v3 f = normalize(sub(tgt, eye));
    v3 rt = normalize(cross(f, up));
    v3 u = cross(rt, f);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < (int64_t)W * H; ++p) {
        int px = (int)(p % W), py = (int)(p / W);
        double sx = (2.0 * (px + 0.5) / W - 1.0) * th * aspect;
        double sy = (1.0 - 2.0 * (py + 0.5) / H) * th;
        v3 d = normalize(add(f, add(scl(rt, sx), scl(u, sy))));
        hit_t h = closest_hit(s, eye, d, 1e30, 0);
        if (tri_out) tri_out[p] = h.tri;
        if (h.tri < 0) {
            for (int c = 0; c < 4; ++c) { pos4[4 * p + c] = 0.0f; nrm4[4 * p + c] = 0.0f; }
            continue;
        }
        v3 n = tri_normal(s, h.tri);
        if (dot(n, d) > 0.0) n = scl(n, -1.0);
        v3 x = add(add(eye, scl(d, h.t)), scl(n, (double)eps));
        pos4[4 * p + 0] = (float)x.x; pos4[4 * p + 1] = (float)x.y;
        pos4[4 * p + 2] = (float)x.z; pos4[4 * p + 3] = 1.0f;
        nrm4[4 * p + 0] = (float)n.x; nrm4[4 * p + 1] = (float)n.y;
        nrm4[4 * p + 2] = (float)n.z; nrm4[4 * p + 3] = 0.0f;
    }
}

/* ----------------------------------------------------------------------------------
 * Step 1 of Algorithms 1 and 2: one ray per receiver.
 *  AO (Eq. 2, Alg. 1): cosine direction about n_x from the receiver point,
 *     t in (0, R].
 *  Shadow (Eq. 5, Alg. 2): y uniform on the light, direction (y - x)/|y - x|,
 *     t in (0, |y - x|].
 * -------------------------------------------------------------------------------- */
static void make_ray(int effect, v3 xh, v3 nx, uint32_t pix, float radius, const light_t* L,
                     uint64_t seed, uint32_t sample, v3* dir, double* tmax) {
    double u1, u2;
    if (effect == 0) {
        rng_pair(seed, pix, sample, ORC_STREAM_AO, &u1, &u2);
        *dir = cosine_dir(nx, u1, u2);
        *tmax = (double)radius;
    } else {
        rng_pair(seed, pix, sample, ORC_STREAM_SHADOW, &u1, &u2);
        v3 y = add(L->c, add(scl(L->eu, u1 - 0.5), scl(L->ev, u2 - 0.5)));
        v3 dv = sub(y, xh);
        double len = sqrt(dot(dv, dv));
        *dir = scl(dv, 1.0 / len);
        *tmax = len;
    }
}

ORC_API void orc_ray(int effect, const float* pos4, const float* nrm4, uint32_t pix, float radius,
                     const float* light, uint64_t seed, uint32_t sample, double out[4]) {
    light_t L;
    if (effect == 1) L = mk_light(light);
    v3 d;
    double tmax;
    make_ray(effect, ldf(pos4), ldf(nrm4), pix, radius, &L, seed, sample, &d, &tmax);
    out[0] = d.x; out[1] = d.y; out[2] = d.z; out[3] = tmax;
}

/* Record layout (8 doubles per pixel): z.xyz, n_z.xyz (oriented toward the
 * source receiver), t, triangle id (-1 = no occluder). */
typedef struct { int x0, y0, x1, y1; } rect_t;

static void trace_px(const scene_t* s, int effect, const float* pos4, const float* nrm4, int64_t p,
                     float radius, const light_t* L, uint64_t seed, uint32_t sample, double* rec,
                     double* margin) {
    double* r = rec + 8 * p;
    if (pos4[4 * p + 3] == 0.0f) {
        for (int c = 0; c < 7; ++c) r[c] = 0.0;
        r[7] = -1.0;
        if (margin) margin[p] = INFINITY;
        return;
    }
    v3 xh = ldf(pos4 + 4 * p), nx = ldf(nrm4 + 4 * p);
    v3 d;
    double tmax;
    make_ray(effect, xh, nx, (uint32_t)p, radius, L, seed, sample, &d, &tmax);
    hit_t h = closest_hit(s, xh, d, tmax, 0);
    if (margin) margin[p] = h.margin;
    if (h.tri < 0) {
        for (int c = 0; c < 7; ++c) r[c] = 0.0;
        r[7] = -1.0;
        return;
    }
    v3 z = add(xh, scl(d, h.t));
    v3 nz = tri_normal(s, h.tri);
    if (dot(nz, d) > 0.0) nz = scl(nz, -1.0);
    r[0] = z.x; r[1] = z.y; r[2] = z.z;
    r[3] = nz.x; r[4] = nz.y; r[5] = nz.z;
    r[6] = h.t;
    r[7] = (double)h.tri;
}

ORC_API void orc_trace(const void* sc, int effect, int W, int H, const float* pos4,
                       const float* nrm4, float radius, const float* light, uint64_t seed,
                       uint32_t sample, int x0, int y0, int w, int h, double* rec, double* margin) {
    const scene_t* s = (const scene_t*)sc;
    light_t L;
    if (effect == 1) L = mk_light(light);
    int64_t n = (int64_t)w * h;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n; ++q) {
        int px = x0 + (int)(q % w), py = y0 + (int)(q / w);
        if (px < 0 || py < 0 || px >= W || py >= H) continue;
        trace_px(s, effect, pos4, nrm4, (int64_t)py * W + px, radius, &L, seed, sample, rec, margin);
    }
}

/* ----------------------------------------------------------------------------------
 * Neighbour sets N_i (Eq. 8).
 *  kind 0 GROUP: the gw x gh block of the screen partition containing i.
 *  kind 1 BOX:   the gw x gh window centred on i (dx in [-(gw-1)/2, gw/2]).
 *  kind 2 OFFSETS: i itself plus i + o_a for the given offsets.
 * Members outside the image or with an invalid G-buffer entry are dropped.
 * -------------------------------------------------------------------------------- */
#define MAX_MEMBERS 64

/* Kind 3 (RANDOM): a neighbour set drawn per receiver, the per-pixel form of N_i in
 * Eq. 8 (the paper's neighbourhoods are per receiver; its random disk sets are not
 * specified further).  Reading: slot s (1 .. n_off) of receiver pixel p takes the first
 * attempt a (0 .. 31) of Philox4x32-10 with counter (p, sample, 2, 32 s + a) and key
 * (seed low, seed high) whose first two words w0, w1 give
 *   dx = floor(w0 (2R + 1) / 2^32) - R,  dy = floor(w1 (2R + 1) / 2^32) - R
 * with dx^2 + dy^2 <= R^2, (dx, dy) != (0, 0) and (dx, dy) not taken by an earlier slot
 * of p; a slot with no such attempt stays empty.  Integer arithmetic only. */
static int random_offset(uint64_t seed, uint32_t pix, uint32_t sample, int slot, int R,
                         const int* acc, int nacc, int* dx, int* dy) {
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int a = 0; a < 32; ++a) {
        uint32_t ctr[4] = {pix, sample, 2u, (uint32_t)(32 * slot + a)}, o[4];
        orc_philox4x32_10(ctr, key, o);
        int x = (int)(((uint64_t)o[0] * (uint64_t)(2 * R + 1)) >> 32) - R;
        int y = (int)(((uint64_t)o[1] * (uint64_t)(2 * R + 1)) >> 32) - R;
        if (x * x + y * y > R * R || (x == 0 && y == 0)) continue;
        int dup = 0;
        for (int q = 0; q < nacc; ++q)
            if (acc[2 * q] == x && acc[2 * q + 1] == y) dup = 1;
        if (dup) continue;
        *dx = x;
        *dy = y;
        return 1;
    }
    return 0;
}

/* The offsets drawn for receiver pixel p (kind 3), in slot order; returns their count. */
ORC_API int orc_random_offsets(uint64_t seed, uint32_t pix, uint32_t sample, int R, int n_off,
                               int32_t* out) {
    int acc[2 * MAX_MEMBERS], nacc = 0;
    for (int s = 1; s <= n_off && s < MAX_MEMBERS; ++s) {
        int dx, dy;
        if (!random_offset(seed, pix, sample, s, R, acc, nacc, &dx, &dy)) continue;
        acc[2 * nacc] = dx;
        acc[2 * nacc + 1] = dy;
        ++nacc;
    }
    for (int q = 0; q < 2 * nacc; ++q) out[q] = acc[q];
    return nacc;
}

static int members(int W, int H, const float* pos4, int px, int py, int kind, int gw, int gh,
                   const int32_t* off, int n_off, uint64_t pseed, uint32_t psample, int64_t* out) {
    int n = 0;
    if (kind == 3) {
        int32_t ro[2 * MAX_MEMBERS];
        int nr = orc_random_offsets(pseed, (uint32_t)((int64_t)py * W + px), psample, gw, n_off, ro);
        for (int a = -1; a < nr; ++a) {
            int x = px + (a < 0 ? 0 : ro[2 * a]), y = py + (a < 0 ? 0 : ro[2 * a + 1]);
            if (x < 0 || y < 0 || x >= W || y >= H) continue;
            int64_t q = (int64_t)y * W + x;
            if (pos4[4 * q + 3] != 0.0f && n < MAX_MEMBERS) out[n++] = q;
        }
        return n;
    }
    if (kind == 0) {
        int bx = (px / gw) * gw, by = (py / gh) * gh;
        for (int y = by; y < by + gh; ++y)
            for (int x = bx; x < bx + gw; ++x) {
                if (x >= W || y >= H) continue;
                int64_t q = (int64_t)y * W + x;
                if (pos4[4 * q + 3] != 0.0f && n < MAX_MEMBERS) out[n++] = q;
            }
    } else if (kind == 1) {
        for (int dy = -(gh - 1) / 2; dy <= gh / 2; ++dy)
            for (int dx = -(gw - 1) / 2; dx <= gw / 2; ++dx) {
                int x = px + dx, y = py + dy;
                if (x < 0 || y < 0 || x >= W || y >= H) continue;
                int64_t q = (int64_t)y * W + x;
                if (pos4[4 * q + 3] != 0.0f && n < MAX_MEMBERS) out[n++] = q;
            }
    } else {
        for (int a = -1; a < n_off; ++a) {
            int x = px + (a < 0 ? 0 : off[2 * a]), y = py + (a < 0 ? 0 : off[2 * a + 1]);
            if (x < 0 || y < 0 || x >= W || y >= H) continue;
            int64_t q = (int64_t)y * W + x;
            if (pos4[4 * q + 3] != 0.0f && n < MAX_MEMBERS) out[n++] = q;
        }
    }
    return n;
}

/* ----------------------------------------------------------------------------------
 * Densities of a candidate z (normal n_z facing its source) at receiver x.
 *
 * AO, Eq. 15 without the first-hit factor:
 *   p(z|x) = (1/pi) <n_x, w_xz> <n_z, w_zx> / |x - z|^2 * 1[|x - z| <= R]
 *          = (1/pi) max(0, n_x.d) max(0, -n_z.d) / r^4,   d = z - x, r^2 = d.d.
 *
 * Shadow, Eqs. 20-21 without the first-hit factor: the ray x + s d meets the
 * light plane at s_L = n_L.(c - x) / n_L.d (needs n_L.d < 0 and s_L > 1);
 * y' = x + s_L d must lie in the rectangle.  With |x - y'| = s_L r and
 * cos_y' = -n_L.d / r, Eq. 20 becomes J = s_L^2 (-n_z.d) / (-n_L.d), and
 * p = J / Area.
 * -------------------------------------------------------------------------------- */
#define SUPPORT_SLACK (1.0 + 1.0 / 65536.0)

static double dens_ao(v3 z, v3 nz, v3 xh, v3 nx, double R2s, double* margin) {
    v3 d = sub(z, xh);
    double r2 = dot(d, d);
    double a = dot(nx, d), b = -dot(nz, d);
    if (a <= 0.0 || b <= 0.0) return 0.0;
    if (margin) *margin = fmin(*margin, fabs(r2 - R2s) / R2s);
    if (!(r2 > 0.0 && r2 <= R2s)) return 0.0;
    return a * b / (M_PI * r2 * r2);
}

static double dens_sh(v3 z, v3 nz, v3 xh, const light_t* L, double* margin) {
    v3 d = sub(z, xh);
    double nd = dot(L->n, d);
    double cz = -dot(nz, d);
    if (!(nd < 0.0) || cz <= 0.0) return 0.0;
    double sL = dot(L->n, sub(L->c, xh)) / nd;
    if (margin) *margin = fmin(*margin, fabs(sL - 1.0));
    if (!(sL > 1.0)) return 0.0;
    v3 q = sub(add(xh, scl(d, sL)), L->c);
    double a = dot(q, L->eu) / L->eu2, b = dot(q, L->ev) / L->ev2;
    double lim = 0.5 * SUPPORT_SLACK;
    if (margin) *margin = fmin(*margin, fmin(fabs(lim - fabs(a)), fabs(lim - fabs(b))) / lim);
    if (fabs(a) > lim || fabs(b) > lim) return 0.0;
    return sL * sL * cz / (-nd) / L->area;
}

/* Biased density of candidate (z, n_z) at receiver (x, n_x): Eq. 15 (AO,
 * effect 0) or Eq. 21 (shadow, effect 1) without the first-hit factor. */
ORC_API double orc_density(int effect, const double* z, const double* nz, const double* x,
                           const double* nx, float radius, const float* light) {
    v3 Z = mk(z[0], z[1], z[2]), NZ = mk(nz[0], nz[1], nz[2]);
    v3 X = mk(x[0], x[1], x[2]), NX = mk(nx[0], nx[1], nx[2]);
    if (effect == 0)
        return dens_ao(Z, NZ, X, NX, (double)radius * (double)radius * SUPPORT_SLACK, NULL);
    light_t L = mk_light(light);
    return dens_sh(Z, NZ, X, &L, NULL);
}

/* First-hit predicate Occ(x, z_j) (Eq. 7): the closest hit of the segment
 * from x toward z_j (direction z_j - x, t in (0, 1 + 2^-10]) is z_j's triangle. */
static int occ_pred(const scene_t* s, v3 xh, v3 z, int64_t tri, double* margin) {
    hit_t h = closest_hit(s, xh, sub(z, xh), 1.0 + 1.0 / 1024.0, 0);
    if (margin) *margin = fmin(*margin, h.margin);
    return h.tri == tri;
}

enum { EST_NOREUSE = 0, EST_BIASED = 1, EST_UNBIASED = 2, EST_BOXMEAN = 3, EST_LIGHT_UNBIASED = 4 };

typedef struct {
    const scene_t* s;
    int effect, W, H;
    const float* pos4;
    const float* nrm4;
    const double* rec;
    int kind, gw, gh, n_off;
    const int32_t* off;
    uint64_t pseed;     /* kind 3: offset-draw key and sample */
    uint32_t psample;
    int estimator;
    double R2s;
    light_t L;
} reuse_args;

static double dens(const reuse_args* a, int64_t j, int64_t k, double* margin) {
    const double* r = a->rec + 8 * j;
    v3 z = mk(r[0], r[1], r[2]), nz = mk(r[3], r[4], r[5]);
    v3 xh = ldf(a->pos4 + 4 * k), nx = ldf(a->nrm4 + 4 * k);
    double p = a->effect == 0 ? dens_ao(z, nz, xh, nx, a->R2s, margin)
                              : dens_sh(z, nz, xh, &a->L, margin);
    if (a->estimator == EST_UNBIASED && p > 0.0 && k != j)
        if (!occ_pred(a->s, xh, z, (int64_t)r[7], margin)) p = 0.0;
    return p;
}

/* Eqs. 17/18 (AO), 23/24 (shadow): out = 1 - sum_j p(z_j|x_i) / sum_k p(z_j|x_k). */
static double reuse_px(const reuse_args* a, int px, int py, double* margin) {
    int64_t i = (int64_t)py * a->W + px;
    *margin = INFINITY;
    if (a->pos4[4 * i + 3] == 0.0f) return 1.0;
    if (a->estimator == EST_NOREUSE) return a->rec[8 * i + 7] < 0.0 ? 1.0 : 0.0;
    int64_t m[MAX_MEMBERS];
    int n = members(a->W, a->H, a->pos4, px, py, a->kind, a->gw, a->gh, a->off, a->n_off,
                    a->pseed, a->psample, m);
    if (a->estimator == EST_BOXMEAN) {
        double v = 0.0;
        for (int q = 0; q < n; ++q) v += a->rec[8 * m[q] + 7] < 0.0 ? 1.0 : 0.0;
        return v / n;
    }
    double B = 0.0;
    int blocked = 0;
    for (int q = 0; q < n; ++q) {
        int64_t j = m[q];
        if (a->rec[8 * j + 7] < 0.0) continue;
        ++blocked;
        double pi = dens(a, j, i, margin);
        if (!(pi > 0.0)) continue;
        double P = 0.0;
        for (int e = 0; e < n; ++e) P += dens(a, j, m[e], margin);
        if (P > 0.0) B += pi / P;
    }
    if (a->effect == 1 && a->estimator == EST_BIASED && blocked == n) return 0.0;
    return 1.0 - B;
}

static reuse_args mk_args(const void* sc, int effect, int W, int H, const float* pos4,
                          const float* nrm4, const double* rec, int kind, int gw, int gh,
                          const int32_t* off, int n_off, uint64_t pseed, uint32_t psample,
                          int estimator, float radius, const float* light) {
    reuse_args a;
    memset(&a, 0, sizeof(a));
    a.s = (const scene_t*)sc;
    a.effect = effect; a.W = W; a.H = H; a.pos4 = pos4; a.nrm4 = nrm4; a.rec = rec;
    a.kind = kind; a.gw = gw; a.gh = gh; a.off = off; a.n_off = n_off;
    a.pseed = pseed; a.psample = psample;
    a.estimator = estimator;
    a.R2s = (double)radius * (double)radius * SUPPORT_SLACK;
    if (effect == 1) a.L = mk_light(light);
    return a;
}

ORC_API void orc_reuse(const void* sc, int effect, int W, int H, const float* pos4,
                       const float* nrm4, const double* rec, int kind, int gw, int gh,
                       const int32_t* off, int n_off, uint64_t pseed, uint32_t psample,
                       int estimator, float radius, const float* light, int x0, int y0, int w,
                       int h, double* out, double* margin) {
    reuse_args a = mk_args(sc, effect, W, H, pos4, nrm4, rec, kind, gw, gh, off, n_off, pseed,
                           psample, estimator, radius, light);
    int64_t n = (int64_t)w * h;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < n; ++q) {
        int px = x0 + (int)(q % w), py = y0 + (int)(q / w);
        if (px < 0 || py < 0 || px >= W || py >= H) continue;
        int64_t i = (int64_t)py * W + px;
        double mg;
        out[i] = reuse_px(&a, px, py, &mg);
        if (margin) margin[i] = mg;
    }
}

/* ----------------------------------------------------------------------------------
 * Unbiased light-sample reuse, Light(N U) of Sec. 6.2 (the comparison baseline for
 * shadows): receiver i re-evaluates the visibility of every member j's light sample y_j
 * (Eq. 5, drawn with j's own random numbers) from its own receiver point.  With the
 * uniform area sampler every member's sample has the same density 1/|A|, so the balance
 * heuristic weighs each of them 1/|N_i| and the estimate of Eq. 4 is the mean visibility
 * of the |N_i| segments x_i -> y_j.  For j = i the segment is i's own step-1 shadow ray.
 * -------------------------------------------------------------------------------- */
static double light_reuse_px(const scene_t* s, int W, int H, const float* pos4, int px, int py,
                             int kind, int gw, int gh, const int32_t* off, int n_off,
                             uint64_t pseed, const light_t* L, uint64_t seed, uint32_t sample,
                             double* margin) {
    int64_t i = (int64_t)py * W + px;
    *margin = INFINITY;
    if (pos4[4 * i + 3] == 0.0f) return 1.0;
    int64_t m[MAX_MEMBERS];
    int n = members(W, H, pos4, px, py, kind, gw, gh, off, n_off, pseed, sample, m);
    v3 xh = ldf(pos4 + 4 * i);
    double vis = 0.0;
    for (int q = 0; q < n; ++q) {
        double u1, u2;
        rng_pair(seed, (uint32_t)m[q], sample, ORC_STREAM_SHADOW, &u1, &u2);
        v3 y = add(L->c, add(scl(L->eu, u1 - 0.5), scl(L->ev, u2 - 0.5)));
        v3 dv = sub(y, xh);
        double len = sqrt(dot(dv, dv));
        hit_t h = closest_hit(s, xh, scl(dv, 1.0 / len), len, 0);
        *margin = fmin(*margin, h.margin);
        if (h.tri < 0) vis += 1.0;
    }
    return vis / n;
}

ORC_API void orc_reuse_light(const void* sc, int W, int H, const float* pos4, int kind, int gw,
                             int gh, const int32_t* off, int n_off, uint64_t pseed,
                             const float* light, uint64_t seed, uint32_t sample, int x0, int y0,
                             int w, int h, double* out, double* margin) {
    const scene_t* s = (const scene_t*)sc;
    light_t L = mk_light(light);
    int64_t n = (int64_t)w * h;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < n; ++q) {
        int px = x0 + (int)(q % w), py = y0 + (int)(q / w);
        if (px < 0 || py < 0 || px >= W || py >= H) continue;
        int64_t i = (int64_t)py * W + px;
        double mg;
        out[i] = light_reuse_px(s, W, H, pos4, px, py, kind, gw, gh, off, n_off, pseed, &L, seed,
                                sample, &mg);
        if (margin) margin[i] = mg;
    }
}

/* Balance-heuristic weights (Eq. 11) seen by receiver i: for every member j
 * with an occluder and every member k, w[j][k] = p(z_j|x_k) / sum_e p(z_j|x_e)
 * (0 when the sum is 0).  Returns the member count; ids go to members_out. */
ORC_API int orc_mis_weights(const void* sc, int effect, int W, int H, const float* pos4,
                            const float* nrm4, const double* rec, int kind, int gw, int gh,
                            const int32_t* off, int n_off, uint64_t pseed, uint32_t psample,
                            int estimator, float radius, const float* light, int px, int py,
                            int64_t* members_out, double* w) {
    reuse_args a = mk_args(sc, effect, W, H, pos4, nrm4, rec, kind, gw, gh, off, n_off, pseed,
                           psample, estimator, radius, light);
    int n = members(W, H, pos4, px, py, kind, gw, gh, off, n_off, pseed, psample, members_out);
    for (int q = 0; q < n; ++q) {
        int64_t j = members_out[q];
        double P = 0.0, p[MAX_MEMBERS];
        for (int e = 0; e < n; ++e) {
            p[e] = a.rec[8 * j + 7] < 0.0 ? 0.0 : dens(&a, j, members_out[e], NULL);
            P += p[e];
        }
        for (int e = 0; e < n; ++e) w[q * n + e] = P > 0.0 ? p[e] / P : 0.0;
    }
    return n;
}

/* ----------------------------------------------------------------------------------
 * M-sample accumulation over a region (per-pixel mean and unbiased variance of
 * the per-sample estimate).  Each sample traces the region plus the halo its
 * neighbour sets reach, then evaluates the estimator (Algorithms 1-2 return
 * 1 - B_i / M: the mean of the per-sample values).
 * -------------------------------------------------------------------------------- */
ORC_API void orc_accumulate(const void* sc, int effect, int W, int H, const float* pos4,
                            const float* nrm4, int kind, int gw, int gh, const int32_t* off,
                            int n_off, uint64_t pseed, int estimator, float radius,
                            const float* light, uint64_t seed, uint32_t sample0, int M, int x0,
                            int y0, int w, int h, double* mean, double* var) {
    int hx0 = x0, hy0 = y0, hx1 = x0 + w, hy1 = y0 + h;
    if (kind == 3) {
        hx0 -= gw; hx1 += gw; hy0 -= gw; hy1 += gw;
    } else if (kind == 0) {
        hx0 = (x0 / gw) * gw; hy0 = (y0 / gh) * gh;
        hx1 = ((x0 + w + gw - 1) / gw) * gw; hy1 = ((y0 + h + gh - 1) / gh) * gh;
    } else if (kind == 1) {
        hx0 -= (gw - 1) / 2; hx1 += gw / 2; hy0 -= (gh - 1) / 2; hy1 += gh / 2;
    } else {
        for (int a = 0; a < n_off; ++a) {
            if (off[2 * a] < 0 && x0 + off[2 * a] < hx0) hx0 = x0 + off[2 * a];
            if (off[2 * a] > 0 && x0 + w + off[2 * a] > hx1) hx1 = x0 + w + off[2 * a];
            if (off[2 * a + 1] < 0 && y0 + off[2 * a + 1] < hy0) hy0 = y0 + off[2 * a + 1];
            if (off[2 * a + 1] > 0 && y0 + h + off[2 * a + 1] > hy1) hy1 = y0 + h + off[2 * a + 1];
        }
    }
    if (hx0 < 0) hx0 = 0;
    if (hy0 < 0) hy0 = 0;
    if (hx1 > W) hx1 = W;
    if (hy1 > H) hy1 = H;
    int64_t P = (int64_t)W * H;
    double* rec = (double*)calloc((size_t)P * 8, sizeof(double));
    double* out = (double*)calloc((size_t)P, sizeof(double));
    for (int64_t i = 0; i < (int64_t)w * h; ++i) { mean[i] = 0.0; var[i] = 0.0; }
    for (int m = 0; m < M; ++m) {
        if (estimator == EST_LIGHT_UNBIASED) {
            orc_reuse_light(sc, W, H, pos4, kind, gw, gh, off, n_off, pseed, light, seed,
                            sample0 + (uint32_t)m, x0, y0, w, h, out, NULL);
        } else {
            orc_trace(sc, effect, W, H, pos4, nrm4, radius, light, seed, sample0 + (uint32_t)m,
                      hx0, hy0, hx1 - hx0, hy1 - hy0, rec, NULL);
            orc_reuse(sc, effect, W, H, pos4, nrm4, rec, kind, gw, gh, off, n_off, pseed,
                      sample0 + (uint32_t)m, estimator, radius, light, x0, y0, w, h, out, NULL);
        }
        for (int64_t q = 0; q < (int64_t)w * h; ++q) {
            int px = x0 + (int)(q % w), py = y0 + (int)(q / w);
            double v = out[(int64_t)py * W + px];
            double delta = v - mean[q];
            mean[q] += delta / (m + 1);
            var[q] += delta * (v - mean[q]);
        }
    }
    for (int64_t q = 0; q < (int64_t)w * h; ++q) var[q] = M > 1 ? var[q] / (M - 1) : 0.0;
    free(rec);
    free(out);
}

ORC_API void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

ORC_API int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
