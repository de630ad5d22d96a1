/*
 * FP64 CPU oracle for plenoctree luminaire rendering.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this code.  It shares nothing with the CUDA
 * library: not a header, not a helper, not a constant.
 *
 * What it computes (paper Sec. 4.1):
 *   L_e(r) = int_0^{t1} T(r,t) sigma(r(t)) Phi(r(t), w) dt      (Eq. 3)
 *   alpha(r) = 1 - T(r, t1)                                      (Eq. 5)
 * with either Beer-Lambert transmittance T = exp(-int sigma) or the linear
 * transmittance T = max(0, 1 - int sigma) (Eq. 4).  In a plenoctree sigma and
 * the SH coefficients are constant inside each leaf (Sec. 4.2, Sec. 5), so
 * the integral is an exact sum over the leaf segments the ray crosses: the
 * oracle enumerates those segments in FP64 (point -> leaf descent, exact
 * dyadic cell planes) and integrates each one in closed form.
 *
 *   exponential: w_i = T_i (1 - exp(-sigma_i dt_i)),  T_{i+1} = exp(-sum sigma dt)
 *   linear     : T_{i+1} = max(0, 1 - sum sigma dt),   w_i = T_i - T_{i+1}
 *                (NeRF-style quadrature weights, which sum to alpha)
 *   linear, literal Eq. 3 with Eq. 4 inside the segment:
 *                w_i = (T_i^2 - T_{i+1}^2) / 2
 *   L_e = sum_i w_i Phi_i,  Phi_i = S(sum_k c_{i,k} Y_k(d))          (Eq. 6)
 *   S = max(0, .) or L_max * sigmoid(.)
 *
 * SH basis: real, orthonormal, index k = l(l+1)+m, m < 0 <-> sin(|m| phi),
 * no Condon-Shortley phase, built from the associated-Legendre recursion and
 * the normalisation constants (Sec. 4.2 names the basis, not a convention).
 *
 * Conventions (readings of the paper):
 *   - the ray is r(t) = o + t d with the caller's march direction d; SH is
 *     evaluated at d (normalised in FP64);
 *   - lookup tie rule: a point exactly on a mid-plane goes to the upper child
 *     when the direction component is >= 0 (or when there is no direction);
 *     the root box is closed;
 *   - after a segment, the exit coordinate(s) are snapped to the exact plane;
 *   - early stop: after a segment, stop if T < t_stop or T <= 0;
 *   - sigma < sigma_min is treated as zero density, and with `saturate` a ray
 *     whose final T is below t_stop counts as opaque (T = 0): the sigma_min /
 *     alpha_max heuristics of Sec. 6 ("Performance vs Quality"), with
 *     t_stop = 1 - alpha_max;
 *   - proxy geometry (Sec. 5, a spherical or a box proxy): the box is the tree's
 *     bounding box; a sphere proxy restricts the integral to the part of the
 *     ray inside both the box and the ball.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t depth, sh_degree;
    int64_t n_nodes, n_leaves;
    const int32_t* child;  /* [n_nodes][8] */
    const float* sigma;    /* [n_leaves] */
    const float* sh;       /* [n_leaves][3][K] */
    double bbox_min[3], bbox_max[3];
} oracle_tree;

typedef struct {
    int32_t transmittance; /* 0 exponential, 1 linear (dT weights), 2 linear literal */
    int32_t activation;    /* 0 max(0,.), 1 l_max * sigmoid(.) */
    double l_max;
    double t_stop;
    double sigma_min;
    int32_t saturate;      /* 1: T = 0 when the final T < t_stop */
    int32_t proxy;         /* 0 box, 1 sphere */
    double sphere[4];      /* sphere proxy: centre xyz and radius, world units */
} oracle_params;

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Real spherical harmonics from the associated Legendre functions.     */

static double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* P_l^m(x), m >= 0, without the Condon-Shortley phase. */
static double assoc_legendre(int l, int m, double x) {
    double pmm = 1.0;
    if (m > 0) {
        double s = sqrt((1.0 - x) * (1.0 + x));
        double f = 1.0;
        for (int i = 1; i <= m; ++i) {
            pmm *= f * s;
            f += 2.0;
        }
    }
    if (l == m) return pmm;
    double pmm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pmm1;
    double pll = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pll = ((2.0 * ll - 1.0) * x * pmm1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pmm1;
        pmm1 = pll;
    }
    return pll;
}

/* Y[k], k = l(l+1)+m, for the direction (dx,dy,dz) (normalised here). */
void oracle_sh_basis(int degree, double dx, double dy, double dz, double* Y) {
    double n = sqrt(dx * dx + dy * dy + dz * dz);
    double x = dx / n, y = dy / n, z = dz / n;
    double phi = atan2(y, x);
    for (int l = 0; l <= degree; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * OR_PI) * factorial(l - am) / factorial(l + am));
            double P = assoc_legendre(l, am, z);
            double v;
            if (m == 0) v = K * P;
            else if (m > 0) v = sqrt(2.0) * K * P * cos(am * phi);
            else v = sqrt(2.0) * K * P * sin(am * phi);
            Y[l * (l + 1) + m] = v;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Point -> leaf.  Returns the leaf id (>= 0), -1 for an empty octant, -2
 * when p is outside the unit cube or the tree is malformed.  Writes the
 * cell's lower corner and edge length. */
static int64_t locate(const oracle_tree* t, const double p[3], const double* dir, double lo[3], double* size,
                      int* level) {
    for (int a = 0; a < 3; ++a)
        if (!(p[a] >= 0.0 && p[a] <= 1.0)) return -2;
    lo[0] = lo[1] = lo[2] = 0.0;
    *size = 1.0;
    *level = 0;
    if (t->n_nodes == 0) return t->n_leaves == 1 ? 0 : -2; /* depth-0 tree: the root is a leaf */
    int64_t node = 0;
    for (int l = 0; l <= t->depth; ++l) {
        int slot = 0;
        double half = *size * 0.5;
        for (int a = 0; a < 3; ++a) {
            double mid = lo[a] + half;
            int up = p[a] > mid || (p[a] == mid && (dir == NULL || dir[a] >= 0.0));
            if (up) lo[a] = mid;
            slot |= up << a;
        }
        *size = half;
        *level = l + 1;
        int32_t e = t->child[node * 8 + slot];
        if (e >= 0) {
            if (e >= t->n_nodes) return -2;
            node = e;
            continue;
        }
        if (e == -1) return -1;
        int64_t leaf = -(int64_t)e - 2;
        return leaf < t->n_leaves ? leaf : -2;
    }
    return -2; /* deeper than the declared depth */
}

void oracle_lookup(const oracle_tree* t, const float* pts, const float* dirs, int64_t n, int64_t* leaf_out,
                   int32_t* level_out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double p[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
        double d[3];
        if (dirs) {
            d[0] = dirs[3 * i];
            d[1] = dirs[3 * i + 1];
            d[2] = dirs[3 * i + 2];
        }
        double lo[3], size;
        int level;
        leaf_out[i] = locate(t, p, dirs ? d : NULL, lo, &size, &level);
        if (level_out) level_out[i] = level;
    }
}

/* ------------------------------------------------------------------ */
/* One ray.  Outputs radiance, transmittance, the per-channel error scale
 * sum_i w_i sum_k |c_k Y_k| (or sum_i w_i Phi_i for the sigmoid), the number
 * of leaf segments and of segments whose SH record is read, and an optional
 * trace of (leaf id or -1, t_in, t_out).  `cond` is the per-channel
 * sensitivity sum_i OD_i |Phi_i| (OD_i = optical depth at the end of segment
 * i): an error e in every optical depth moves the linear-model radiance by at
 * most e * cond.  Status: 0 ok, 1 iteration cap,
 * 2 lookup failure, 3 invalid ray (NaN/Inf component or zero direction). */
typedef struct {
    double rgb[3], T, bound[3], cond[3];
    int32_t n_leaf, n_sh, n_cell, status;
} ray_result;

static void render_one(const oracle_tree* t, const oracle_params* prm, const float* ray, ray_result* res,
                       int64_t* tr_leaf, double* tr_t, int32_t tr_max, int32_t* tr_n) {
    const int K = (t->sh_degree + 1) * (t->sh_degree + 1);
    double ext[3], o[3], d[3], dw[3];
    for (int a = 0; a < 3; ++a) {
        ext[a] = t->bbox_max[a] - t->bbox_min[a];
        o[a] = ((double)ray[a] - t->bbox_min[a]) / ext[a];
        dw[a] = ray[3 + a];
        d[a] = dw[a] / ext[a];
    }
    memset(res, 0, sizeof(*res));
    res->T = 1.0;
    if (tr_n) *tr_n = 0;
    /* a ray with a non-finite component or a zero direction is invalid */
    int bad = dw[0] == 0.0 && dw[1] == 0.0 && dw[2] == 0.0;
    for (int a = 0; a < 6; ++a) bad |= !isfinite((double)ray[a]);
    if (bad) {
        res->status = 3;
        res->rgb[0] = res->rgb[1] = res->rgb[2] = res->T = NAN;
        return;
    }

    /* proxy clip: slab test against the unit cube */
    double tn = -INFINITY, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < 0.0 || o[a] > 1.0) return;
            continue;
        }
        double t0 = (0.0 - o[a]) / d[a], t1 = (1.0 - o[a]) / d[a];
        if (t0 > t1) { double s = t0; t0 = t1; t1 = s; }
        if (t0 > tn) tn = t0;
        if (t1 < tf) tf = t1;
    }
    if (!(tn < tf) || !(tf > 0.0)) return;
    if (prm->proxy == 1) {
        /* |o + t d - c|^2 = r^2 in unit-cube coordinates (the box is a cube,
         * so the ball stays a ball) */
        double c[3], b = 0.0, a2 = 0.0, q = 0.0;
        const double r = prm->sphere[3] / ext[0];
        for (int a = 0; a < 3; ++a) {
            c[a] = (prm->sphere[a] - t->bbox_min[a]) / ext[a];
            a2 += d[a] * d[a];
            b += (o[a] - c[a]) * d[a];
            q += (o[a] - c[a]) * (o[a] - c[a]);
        }
        double disc = b * b - a2 * (q - r * r);
        if (!(disc > 0.0)) return;
        double ts0 = (-b - sqrt(disc)) / a2, ts1 = (-b + sqrt(disc)) / a2;
        if (ts0 > tn) tn = ts0;
        if (ts1 < tf) tf = ts1;
        if (!(tn < tf) || !(tf > 0.0)) return;
    }

    double Y[25];
    oracle_sh_basis(t->sh_degree, dw[0], dw[1], dw[2], Y);

    double tcur = tn > 0.0 ? tn : 0.0;
    double p[3];
    for (int a = 0; a < 3; ++a) p[a] = o[a] + tcur * d[a];
    if (tn > 0.0) {
        /* snap the entry face(s) */
        for (int a = 0; a < 3; ++a) {
            if (d[a] == 0.0) continue;
            double t0 = (0.0 - o[a]) / d[a], t1 = (1.0 - o[a]) / d[a];
            double near = t0 < t1 ? t0 : t1;
            if (near == tn) p[a] = d[a] > 0.0 ? 0.0 : 1.0;
        }
    }

    double T = 1.0, od = 0.0;
    const int64_t max_iter = 3 * ((int64_t)1 << t->depth) + 16;
    int64_t iter = 0;
    for (;;) {
        if (++iter > max_iter) { res->status = 1; break; }
        for (int a = 0; a < 3; ++a) { /* FP64 rounding guard for non-snapped coordinates */
            if (p[a] < 0.0) p[a] = 0.0;
            if (p[a] > 1.0) p[a] = 1.0;
        }
        double lo[3], size;
        int level;
        int64_t leaf = locate(t, p, d, lo, &size, &level);
        if (leaf == -2) { res->status = 2; break; }
        double tx[3], tnext = tf;
        for (int a = 0; a < 3; ++a) {
            if (d[a] > 0.0) tx[a] = (lo[a] + size - o[a]) / d[a];
            else if (d[a] < 0.0) tx[a] = (lo[a] - o[a]) / d[a];
            else tx[a] = INFINITY;
            if (tx[a] < tnext) tnext = tx[a];
        }
        double dt = tnext - tcur;
        if (dt < 0.0) dt = 0.0;
        res->n_cell++;
        if (tr_n && *tr_n < tr_max) {
            tr_leaf[*tr_n] = leaf;
            tr_t[2 * *tr_n] = tcur;
            tr_t[2 * *tr_n + 1] = tnext;
            ++*tr_n;
        }
        if (leaf >= 0) {
            res->n_leaf++;
            double sg = t->sigma[leaf];
            if (sg < prm->sigma_min) sg = 0.0;
            if (sg > 0.0) {
                const float* rec = t->sh + (size_t)leaf * 3 * K;
                int emits = 0;
                for (int k = 0; k < 3 * K; ++k) emits |= rec[k] != 0.0f;
                double a_seg = sg * dt, w, Tn;
                if (prm->transmittance == 0) {
                    w = T * (-expm1(-a_seg));
                    od += a_seg;
                    Tn = exp(-od);
                } else {
                    od += a_seg;
                    Tn = 1.0 - od;
                    if (Tn < 0.0) Tn = 0.0;
                    w = prm->transmittance == 1 ? T - Tn : 0.5 * (T * T - Tn * Tn);
                }
                if (emits) res->n_sh++;
                if (emits || prm->activation == 1) {
                    for (int ch = 0; ch < 3; ++ch) {
                        double s = 0.0, sa = 0.0;
                        for (int k = 0; k < K; ++k) {
                            s += rec[ch * K + k] * Y[k];
                            sa += fabs(rec[ch * K + k] * Y[k]);
                        }
                        double c;
                        if (prm->activation == 0) {
                            c = s > 0.0 ? s : 0.0;
                            res->bound[ch] += w * sa;
                            res->cond[ch] += od * sa;
                        } else {
                            c = prm->l_max / (1.0 + exp(-s));
                            res->bound[ch] += w * c;
                            res->cond[ch] += od * c;
                        }
                        res->rgb[ch] += w * c;
                    }
                }
                T = Tn;
            }
        }
        if (tnext >= tf) break;
        if (T < prm->t_stop || T <= 0.0) break;
        /* the exit point lies on the closed box of the cell just left: exit
         * axes on their plane, the others clamped into the box (FP64 rounding
         * of o + t d may put them a hair inside the old cell otherwise) */
        tcur = tnext;
        for (int a = 0; a < 3; ++a) {
            if (tx[a] == tnext) {
                p[a] = d[a] > 0.0 ? lo[a] + size : lo[a];
            } else {
                p[a] = o[a] + tcur * d[a];
                if (p[a] < lo[a]) p[a] = lo[a];
                if (p[a] > lo[a] + size) p[a] = lo[a] + size;
            }
        }
    }
    if (prm->saturate && T < prm->t_stop) T = 0.0;
    res->T = T;
}

/* Render n rays (float[n][6]: origin, direction).  Any output pointer may be
 * NULL.  n_threads <= 0 uses the OpenMP default.  Returns the number of rays
 * whose status is non-zero. */
int64_t oracle_render(const oracle_tree* t, const float* rays, int64_t n, const oracle_params* prm, double* rgb,
                      double* T, double* bound, double* cond, int32_t* n_leaf, int32_t* n_sh, int32_t* n_cell,
                      int32_t* status, int n_threads) {
    int64_t bad = 0;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(n_threads) reduction(+ : bad)
#endif
    for (int64_t i = 0; i < n; ++i) {
        ray_result r;
        render_one(t, prm, rays + 6 * i, &r, NULL, NULL, 0, NULL);
        if (rgb) for (int c = 0; c < 3; ++c) rgb[3 * i + c] = r.rgb[c];
        if (T) T[i] = r.T;
        if (bound) for (int c = 0; c < 3; ++c) bound[3 * i + c] = r.bound[c];
        if (cond) for (int c = 0; c < 3; ++c) cond[3 * i + c] = r.cond[c];
        if (n_leaf) n_leaf[i] = r.n_leaf;
        if (n_sh) n_sh[i] = r.n_sh;
        if (n_cell) n_cell[i] = r.n_cell;
        if (status) status[i] = r.status;
        bad += r.status != 0;
    }
    return bad;
}

/* The ordered cells one ray crosses: leaf id (or -1 for an empty octant) and
 * [t_in, t_out].  Returns the number written (<= max). */
int32_t oracle_trace(const oracle_tree* t, const oracle_params* prm, const float* ray, int32_t max, int64_t* leaf,
                     double* t_in_out) {
    ray_result r;
    int32_t n = 0;
    render_one(t, prm, ray, &r, leaf, t_in_out, max, &n);
    return n;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* The luminaire as an emitter in a path tracer (Sec. 3 Eq. 2, Sec. 5   */
/* "Sampling").  One path per call, FP64, random numbers passed in.     */
/*   camera: pinhole, pixel (px + u0, py + u1);                          */
/*   per bounce b (uniforms u[2+5b .. 6+5b]):                            */
/*     luminaire along the ray: camera rays add L_e, the throughput is   */
/*       multiplied by T (light from behind passes through);             */
/*     wall hit x (room seen from inside), inward normal n, albedo rho;  */
/*     next event: y uniform on the proxy box surface (face by area, then */
/*       uniform on it); if y's face faces x, add                         */
/*       thr rho/pi L_e(x -> y) cos_x cos_y / |y-x|^2 A;                   */
/*     cosine-weighted bounce about n, thr *= rho.                        */
/* emitter 0 queries the tree; emitter 1 is an opaque box of constant     */
/* radiance (the comparison emitter).                                     */

typedef struct {
    double room_min[3], room_max[3];
    double albedo[6][3];
    double cam_pos[3], cam_target[3], cam_up[3];
    double fov_y;
    int32_t width, height, max_bounces, emitter;
    double box_radiance[3];
} oracle_pt_scene;

static void pt_luminaire(const oracle_tree* t, const oracle_params* prm, const oracle_pt_scene* sc,
                         const double o[3], const double d[3], double Le[3], double* T) {
    if (sc->emitter == 1) {
        double tn = -INFINITY, tf = INFINITY;
        int miss = 0;
        for (int a = 0; a < 3; ++a) {
            if (d[a] == 0.0) {
                if (o[a] < t->bbox_min[a] || o[a] > t->bbox_max[a]) miss = 1;
                continue;
            }
            double t0 = (t->bbox_min[a] - o[a]) / d[a], t1 = (t->bbox_max[a] - o[a]) / d[a];
            if (t0 > t1) { double s = t0; t0 = t1; t1 = s; }
            if (t0 > tn) tn = t0;
            if (t1 < tf) tf = t1;
        }
        int hit = !miss && tn < tf && tf > 0.0;
        for (int c = 0; c < 3; ++c) Le[c] = hit ? sc->box_radiance[c] : 0.0;
        *T = hit ? 0.0 : 1.0;
        return;
    }
    float ray[6];
    for (int a = 0; a < 3; ++a) {
        ray[a] = (float)o[a];
        ray[3 + a] = (float)d[a];
    }
    ray_result r;
    render_one(t, prm, ray, &r, NULL, NULL, 0, NULL);
    for (int c = 0; c < 3; ++c) Le[c] = r.rgb[c];
    *T = r.T;
}

static void pt_norm(double* v) {
    double s = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= s; v[1] /= s; v[2] /= s;
}

void oracle_pt_sample(const oracle_tree* t, const oracle_params* prm, const oracle_pt_scene* sc, const double* u,
                      int32_t px, int32_t py, double out[3]) {
    double fwd[3], right[3], up[3], o[3], d[3], thr[3] = {1.0, 1.0, 1.0}, L[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) fwd[k] = sc->cam_target[k] - sc->cam_pos[k];
    pt_norm(fwd);
    right[0] = fwd[1] * sc->cam_up[2] - fwd[2] * sc->cam_up[1];
    right[1] = fwd[2] * sc->cam_up[0] - fwd[0] * sc->cam_up[2];
    right[2] = fwd[0] * sc->cam_up[1] - fwd[1] * sc->cam_up[0];
    pt_norm(right);
    up[0] = right[1] * fwd[2] - right[2] * fwd[1];
    up[1] = right[2] * fwd[0] - right[0] * fwd[2];
    up[2] = right[0] * fwd[1] - right[1] * fwd[0];
    double th = tan(0.5 * sc->fov_y);
    double sx = (2.0 * (px + u[0]) / sc->width - 1.0) * th * sc->width / sc->height;
    double sy = (1.0 - 2.0 * (py + u[1]) / sc->height) * th;
    for (int k = 0; k < 3; ++k) {
        o[k] = sc->cam_pos[k];
        d[k] = fwd[k] + sx * right[k] + sy * up[k];
    }
    pt_norm(d);
    double ext[3], area = 0.0, fa[6];
    for (int k = 0; k < 3; ++k) ext[k] = t->bbox_max[k] - t->bbox_min[k];
    for (int f = 0; f < 6; ++f) {
        fa[f] = ext[((f >> 1) + 1) % 3] * ext[((f >> 1) + 2) % 3];
        area += fa[f];
    }
    for (int b = 0; b < sc->max_bounces; ++b) {
        const double* ub = u + 2 + 5 * b;
        double Le[3], T;
        pt_luminaire(t, prm, sc, o, d, Le, &T);
        for (int c = 0; c < 3; ++c) {
            if (b == 0) L[c] += thr[c] * Le[c];
            thr[c] *= T;
        }
        double tw = INFINITY;
        int ax = 0;
        for (int k = 0; k < 3; ++k) {
            if (d[k] == 0.0) continue;
            double tt = ((d[k] > 0.0 ? sc->room_max[k] : sc->room_min[k]) - o[k]) / d[k];
            if (tt < tw) { tw = tt; ax = k; }
        }
        int wall = 2 * ax + (d[ax] > 0.0 ? 1 : 0);
        double x[3], n[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 3; ++k) x[k] = o[k] + tw * d[k];
        x[ax] = d[ax] > 0.0 ? sc->room_max[ax] : sc->room_min[ax];
        n[ax] = d[ax] > 0.0 ? -1.0 : 1.0;
        /* next event toward a uniform point of the proxy surface */
        double acc = 0.0;
        int f = 0;
        for (f = 0; f < 5; ++f) {
            acc += fa[f] / area;
            if (ub[0] < acc) break;
        }
        int fa_ = f >> 1, fb = (fa_ + 1) % 3, fc = (fa_ + 2) % 3;
        double y[3];
        y[fa_] = (f & 1) ? t->bbox_max[fa_] : t->bbox_min[fa_];
        y[fb] = t->bbox_min[fb] + ub[1] * ext[fb];
        y[fc] = t->bbox_min[fc] + ub[2] * ext[fc];
        double w[3];
        for (int k = 0; k < 3; ++k) w[k] = y[k] - x[k];
        double dist2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
        pt_norm(w);
        int faces = (f & 1) ? x[fa_] > y[fa_] : x[fa_] < y[fa_];
        double cos_x = n[0] * w[0] + n[1] * w[1] + n[2] * w[2];
        double cos_y = fabs(w[fa_]);
        if (faces && cos_x > 0.0) {
            double Le2[3], T2;
            pt_luminaire(t, prm, sc, x, w, Le2, &T2);
            double g = cos_x * cos_y / dist2 * area / OR_PI;
            for (int c = 0; c < 3; ++c) L[c] += thr[c] * sc->albedo[wall][c] * g * Le2[c];
        }
        /* cosine-weighted bounce */
        double r = sqrt(ub[3]), phi = 2.0 * OR_PI * ub[4];
        double nd[3];
        nd[ax] = n[ax] * sqrt(fmax(0.0, 1.0 - ub[3]));
        nd[(ax + 1) % 3] = r * cos(phi);
        nd[(ax + 2) % 3] = r * sin(phi);
        for (int k = 0; k < 3; ++k) {
            o[k] = x[k];
            d[k] = nd[k];
            thr[k] *= sc->albedo[wall][k];
        }
    }
    for (int c = 0; c < 3; ++c) out[c] = L[c];
}

/* n paths: path p uses uniforms u[p*dims ..], pixel p % (width*height). */
void oracle_pt_render(const oracle_tree* t, const oracle_params* prm, const oracle_pt_scene* sc, const double* u,
                      int64_t n_paths, int n_threads, double* out) {
    const int dims = 2 + 5 * sc->max_bounces;
    const int64_t pixels = (int64_t)sc->width * sc->height;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(n_threads)
#endif
    for (int64_t p = 0; p < n_paths; ++p) {
        int64_t pix = p % pixels;
        oracle_pt_sample(t, prm, sc, u + p * dims, (int32_t)(pix % sc->width), (int32_t)(pix / sc->width), out + 3 * p);
    }
}
