/*
 * Seeded synthetic inputs: a procedural luminaire octree in the canonical
 * host tree format, and ray sets.
 *
 * This module is the only code shared by the FP64 oracle and the CUDA path.
 * It holds none of the rendering method's arithmetic: it decides which cells
 * of a procedural shape are occupied and draws per-leaf values and rays from
 * a counter-based generator.  Nothing here integrates radiance, evaluates
 * spherical harmonics or walks the tree along a ray.
 *
 * Stand-in for the paper's Mitsuba luminaires (Sec. 6.1): a helical emissive
 * coil inside a spherical glass-like shell, voxelised at depth D, with leaf
 * values drawn as the workload description states (sigma log-uniform,
 * SH DC log-uniform per channel, higher bands normal with std 0.1*DC, a
 * Bernoulli fraction of leaves with zero emission).
 *
 * Canonical tree format (shared with the library's plo_tree_desc):
 *   child[n_nodes][8] int32: >= 0 internal node id, -1 empty octant,
 *                            <= -2 leaf, leaf id = -c - 2.
 *   slot = bx | by << 1 | bz << 2, b = 1 for the upper half along that axis.
 *   node 0 is the root, covering the unit cube [0,1]^3.
 *   sigma[n_leaves], sh[n_leaves][3][K], K = (sh_degree + 1)^2.
 *
 * Portability: compiled with -ffp-contract=off; the random stream is pure
 * integer arithmetic, so the same seed gives the same bits on x86-64 and
 * aarch64 up to libm's log/sin/cos/sqrt rounding in the value transforms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define PLOGEN_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Counter-based random numbers: SplitMix64 finaliser (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", 2014) applied to
 * a key built from (seed, stream, index, counter).                     */
static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t rng_u64(uint64_t seed, uint64_t stream, uint64_t index, uint64_t ctr) {
    uint64_t k = mix64(seed ^ mix64(stream * 0xD1B54A32D192ED03ULL + 1));
    k = mix64(k ^ index);
    return mix64(k ^ (ctr * 0x8CB92BA72F3D8DD7ULL + 0x632BE59BD9B4E019ULL));
}
/* uniform in [0,1) with 53 random bits */
static inline double rng_unif(uint64_t seed, uint64_t stream, uint64_t index, uint64_t ctr) {
    return (double)(rng_u64(seed, stream, index, ctr) >> 11) * (1.0 / 9007199254740992.0);
}
/* standard normal (Box-Muller, first output) */
static inline double rng_normal(uint64_t seed, uint64_t stream, uint64_t index, uint64_t ctr) {
    double u1 = rng_unif(seed, stream, index, 2 * ctr);
    double u2 = rng_unif(seed, stream, index, 2 * ctr + 1);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * PLOGEN_PI * u2);
}

enum { STREAM_EMISSIVE = 1, STREAM_SIGMA = 2, STREAM_SH = 3, STREAM_RAY = 4 };

/* ------------------------------------------------------------------ */
typedef struct {
    int32_t depth;          /* 1..16 */
    int32_t sh_degree;      /* 0..4 */
    uint64_t seed;
    double shell_center[3];
    double shell_radius;
    double shell_half_thickness;
    double coil_center_xy[2];
    double coil_radius;       /* helix radius R */
    double coil_tube_radius;  /* tube radius around the helix */
    double coil_z0, coil_z1;  /* slab the coil occupies */
    double coil_turns;        /* pitch = (z1 - z0) / turns */
    double emissive_fraction; /* probability that a leaf emits */
    double sigma_log10_min, sigma_log10_max;
    double dc_log10_min, dc_log10_max;
    double band_rel_std;      /* std of l >= 1 coefficients, relative to the DC */
} plogen_params;

typedef struct {
    plogen_params p;
    int32_t* child;      /* [cap_nodes][8] */
    int64_t n_nodes, cap_nodes;
    uint64_t* leaf_key;  /* packed integer coords of each leaf at level depth */
    int64_t n_leaves, cap_leaves;
} plogen_tree;

static double shell_dist(const plogen_params* p, double x, double y, double z) {
    double dx = x - p->shell_center[0], dy = y - p->shell_center[1], dz = z - p->shell_center[2];
    return fabs(sqrt(dx * dx + dy * dy + dz * dz) - p->shell_radius);
}

/* Distance from (x,y,z) to the nearest point of the infinite helix that
 * shares its azimuth.  It bounds the Euclidean distance to the helix from
 * above and is within 0.3% of it near the tube for the pitches used. */
static double coil_dist(const plogen_params* p, double x, double y, double z) {
    double dx = x - p->coil_center_xy[0], dy = y - p->coil_center_xy[1];
    double rho = sqrt(dx * dx + dy * dy);
    double phi = atan2(dy, dx);
    if (phi < 0) phi += 2.0 * PLOGEN_PI;
    double pitch = (p->coil_z1 - p->coil_z0) / p->coil_turns;
    double u = (z - p->coil_z0) / pitch - phi / (2.0 * PLOGEN_PI);
    double k0 = floor(u + 0.5);
    double best = 1e300;
    for (int j = -1; j <= 1; ++j) {
        double zk = p->coil_z0 + pitch * (phi / (2.0 * PLOGEN_PI) + k0 + j);
        double dr = rho - p->coil_radius, dz = z - zk;
        double d = sqrt(dr * dr + dz * dz);
        if (d < best) best = d;
    }
    return best;
}

static int occupied_point(const plogen_params* p, double x, double y, double z) {
    if (shell_dist(p, x, y, z) <= p->shell_half_thickness) return 1;
    if (z >= p->coil_z0 && z <= p->coil_z1 && coil_dist(p, x, y, z) <= p->coil_tube_radius) return 1;
    return 0;
}

/* Conservative: returns 1 whenever some finest-level cell centre inside the
 * cell may be occupied (shell distance is 1-Lipschitz; the coil distance is
 * given a 1.5x margin). */
static int may_contain(const plogen_params* p, int level, uint32_t cx, uint32_t cy, uint32_t cz) {
    double size = ldexp(1.0, -level);
    double x = (cx + 0.5) * size, y = (cy + 0.5) * size, z = (cz + 0.5) * size;
    double hd = 0.8660254037844387 * size;
    if (shell_dist(p, x, y, z) <= p->shell_half_thickness + hd * 1.0001 + 1e-12) return 1;
    double zlo = cz * size, zhi = zlo + size;
    if (zhi >= p->coil_z0 && zlo <= p->coil_z1 &&
        coil_dist(p, x, y, z) <= p->coil_tube_radius + 1.5 * hd + 1e-12)
        return 1;
    return 0;
}

static int grow_nodes(plogen_tree* t) {
    if (t->n_nodes < t->cap_nodes) return 0;
    int64_t cap = t->cap_nodes ? t->cap_nodes * 2 : 1024;
    int32_t* c = (int32_t*)realloc(t->child, (size_t)cap * 8 * sizeof(int32_t));
    if (!c) return -1;
    t->child = c;
    t->cap_nodes = cap;
    return 0;
}
static int grow_leaves(plogen_tree* t) {
    if (t->n_leaves < t->cap_leaves) return 0;
    int64_t cap = t->cap_leaves ? t->cap_leaves * 2 : 4096;
    uint64_t* k = (uint64_t*)realloc(t->leaf_key, (size_t)cap * sizeof(uint64_t));
    if (!k) return -1;
    t->leaf_key = k;
    t->cap_leaves = cap;
    return 0;
}

/* Fills node `id` (at `level`, integer coords c*) depth-first.  Returns the
 * number of non-empty children, or -1 on allocation failure. */
static int build_node(plogen_tree* t, int64_t id, int level, uint32_t cx, uint32_t cy, uint32_t cz) {
    const plogen_params* p = &t->p;
    int nonempty = 0;
    for (int slot = 0; slot < 8; ++slot) {
        uint32_t x = 2 * cx + (slot & 1), y = 2 * cy + ((slot >> 1) & 1), z = 2 * cz + ((slot >> 2) & 1);
        int cl = level + 1;
        int32_t entry = -1;
        if (cl == p->depth) {
            double size = ldexp(1.0, -cl);
            if (occupied_point(p, (x + 0.5) * size, (y + 0.5) * size, (z + 0.5) * size)) {
                if (grow_leaves(t)) return -1;
                int64_t leaf = t->n_leaves++;
                t->leaf_key[leaf] = (uint64_t)x | ((uint64_t)y << 16) | ((uint64_t)z << 32);
                entry = (int32_t)(-leaf - 2);
            }
        } else if (may_contain(p, cl, x, y, z)) {
            if (grow_nodes(t)) return -1;
            int64_t cid = t->n_nodes++;
            int r = build_node(t, cid, cl, x, y, z);
            if (r < 0) return -1;
            if (r == 0) {
                t->n_nodes = cid; /* subtree was empty: it is the tail, drop it */
            } else {
                entry = (int32_t)cid;
            }
        }
        t->child[id * 8 + slot] = entry;
        if (entry != -1) ++nonempty;
    }
    return nonempty;
}

void plogen_free(plogen_tree* t) {
    if (!t) return;
    free(t->child);
    free(t->leaf_key);
    free(t);
}

/* Pass 1: structure.  Returns NULL on invalid parameters or allocation
 * failure. */
plogen_tree* plogen_build(const plogen_params* p, int64_t* n_nodes, int64_t* n_leaves) {
    if (!p || p->depth < 1 || p->depth > 16 || p->sh_degree < 0 || p->sh_degree > 4) return NULL;
    plogen_tree* t = (plogen_tree*)calloc(1, sizeof(plogen_tree));
    if (!t) return NULL;
    t->p = *p;
    if (grow_nodes(t)) { plogen_free(t); return NULL; }
    t->n_nodes = 1;
    if (build_node(t, 0, 0, 0, 0, 0) < 0) { plogen_free(t); return NULL; }
    *n_nodes = t->n_nodes;
    *n_leaves = t->n_leaves;
    return t;
}

/* Pass 2: copy the child table and draw leaf values into caller buffers:
 * child[n_nodes*8], sigma[n_leaves], sh[n_leaves*3*K] (may be NULL to skip),
 * leaf_xyz[n_leaves*3] integer coords at level depth (may be NULL). */
int plogen_fill(const plogen_tree* t, int32_t* child, float* sigma, float* sh, int32_t* leaf_xyz) {
    const plogen_params* p = &t->p;
    const int K = (p->sh_degree + 1) * (p->sh_degree + 1);
    memcpy(child, t->child, (size_t)t->n_nodes * 8 * sizeof(int32_t));
    const uint64_t seed = p->seed;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < t->n_leaves; ++i) {
        uint64_t key = t->leaf_key[i];
        if (leaf_xyz) {
            leaf_xyz[3 * i + 0] = (int32_t)(key & 0xFFFF);
            leaf_xyz[3 * i + 1] = (int32_t)((key >> 16) & 0xFFFF);
            leaf_xyz[3 * i + 2] = (int32_t)((key >> 32) & 0xFFFF);
        }
        double us = rng_unif(seed, STREAM_SIGMA, key, 0);
        double ls = p->sigma_log10_min + (p->sigma_log10_max - p->sigma_log10_min) * us;
        sigma[i] = (float)pow(10.0, ls);
        if (!sh) continue;
        float* rec = sh + (size_t)i * 3 * K;
        int emits = rng_unif(seed, STREAM_EMISSIVE, key, 0) < p->emissive_fraction;
        for (int ch = 0; ch < 3; ++ch) {
            if (!emits) {
                for (int k = 0; k < K; ++k) rec[ch * K + k] = 0.0f;
                continue;
            }
            double ud = rng_unif(seed, STREAM_SH, key, (uint64_t)ch * 64);
            double dc = pow(10.0, p->dc_log10_min + (p->dc_log10_max - p->dc_log10_min) * ud);
            rec[ch * K + 0] = (float)dc;
            for (int k = 1; k < K; ++k)
                rec[ch * K + k] = (float)(p->band_rel_std * dc * rng_normal(seed, STREAM_SH, key, (uint64_t)ch * 64 + k));
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Rays, written as float[n][6] = origin xyz, unit direction xyz.        */

/* Origins uniform on a sphere of radius `radius` about `center`, each aimed
 * at a uniform point of the unit cube. */
void plogen_rays_sphere(uint64_t seed, int64_t n, const double center[3], double radius, float* rays) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double u = 2.0 * rng_unif(seed, STREAM_RAY, (uint64_t)i, 0) - 1.0;
        double ph = 2.0 * PLOGEN_PI * rng_unif(seed, STREAM_RAY, (uint64_t)i, 1);
        double s = sqrt(fmax(0.0, 1.0 - u * u));
        double o[3] = {center[0] + radius * s * cos(ph), center[1] + radius * s * sin(ph), center[2] + radius * u};
        double tgt[3] = {rng_unif(seed, STREAM_RAY, (uint64_t)i, 2), rng_unif(seed, STREAM_RAY, (uint64_t)i, 3),
                         rng_unif(seed, STREAM_RAY, (uint64_t)i, 4)};
        double d[3] = {tgt[0] - o[0], tgt[1] - o[1], tgt[2] - o[2]};
        double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int a = 0; a < 3; ++a) {
            rays[6 * i + a] = (float)o[a];
            rays[6 * i + 3 + a] = (float)(d[a] / len);
        }
    }
}

/* Rejection helper: does the FP64 ray meet the box [lo,hi] with a
 * positive-length intersection in front of the origin? */
static int meets_box(const double o[3], const double d[3], const double lo[3], const double hi[3]) {
    double tn = -1e300, tf = 1e300;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < lo[a] || o[a] > hi[a]) return 0;
            continue;
        }
        double t1 = (lo[a] - o[a]) / d[a], t2 = (hi[a] - o[a]) / d[a];
        if (t1 > t2) { double tmp = t1; t1 = t2; t2 = tmp; }
        if (t1 > tn) tn = t1;
        if (t2 < tf) tf = t2;
    }
    return tn < tf && tf > 0.0;
}

/* Origins uniform in the room box [room_lo, room_hi] but outside the target
 * box [box_lo, box_hi]; directions cosine-weighted about the unit vector from
 * the origin to the target box centre; each ray index retries with fresh
 * counters until its ray meets the target box.  Returns the total number of
 * attempts (for reporting the acceptance rate), or -1 if some ray exceeded
 * `max_attempts`. */
int64_t plogen_rays_room(uint64_t seed, int64_t n, const double room_lo[3], const double room_hi[3],
                         const double box_lo[3], const double box_hi[3], int64_t max_attempts, float* rays) {
    int64_t total = 0;
    int failed = 0;
    double ctr[3] = {0.5 * (box_lo[0] + box_hi[0]), 0.5 * (box_lo[1] + box_hi[1]), 0.5 * (box_lo[2] + box_hi[2])};
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : total) reduction(| : failed)
    for (int64_t i = 0; i < n; ++i) {
        int64_t a;
        for (a = 0; a < max_attempts; ++a) {
            uint64_t c0 = (uint64_t)a * 8;
            double o[3];
            for (int k = 0; k < 3; ++k)
                o[k] = room_lo[k] + (room_hi[k] - room_lo[k]) * rng_unif(seed, STREAM_RAY, (uint64_t)i, c0 + k);
            if (o[0] >= box_lo[0] && o[0] <= box_hi[0] && o[1] >= box_lo[1] && o[1] <= box_hi[1] &&
                o[2] >= box_lo[2] && o[2] <= box_hi[2])
                continue;
            double w[3] = {ctr[0] - o[0], ctr[1] - o[1], ctr[2] - o[2]};
            double wl = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            for (int k = 0; k < 3; ++k) w[k] /= wl;
            /* orthonormal frame (Frisvad-style, with the singular case flipped) */
            double u[3], v[3];
            if (w[2] < -0.9999999) {
                u[0] = 0; u[1] = -1; u[2] = 0;
                v[0] = -1; v[1] = 0; v[2] = 0;
            } else {
                double a1 = 1.0 / (1.0 + w[2]), b1 = -w[0] * w[1] * a1;
                u[0] = 1.0 - w[0] * w[0] * a1; u[1] = b1; u[2] = -w[0];
                v[0] = b1; v[1] = 1.0 - w[1] * w[1] * a1; v[2] = -w[1];
            }
            double u1 = rng_unif(seed, STREAM_RAY, (uint64_t)i, c0 + 3);
            double u2 = rng_unif(seed, STREAM_RAY, (uint64_t)i, c0 + 4);
            double r = sqrt(u1), ph = 2.0 * PLOGEN_PI * u2;
            double lx = r * cos(ph), ly = r * sin(ph), lz = sqrt(fmax(0.0, 1.0 - u1));
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = lx * u[k] + ly * v[k] + lz * w[k];
            double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int k = 0; k < 3; ++k) d[k] /= dl;
            /* decide on the FP32-rounded ray that is actually emitted */
            float of[3], df[3];
            double od[3], dd[3];
            for (int k = 0; k < 3; ++k) {
                of[k] = (float)o[k]; df[k] = (float)d[k];
                od[k] = of[k]; dd[k] = df[k];
            }
            if (!meets_box(od, dd, box_lo, box_hi)) continue;
            for (int k = 0; k < 3; ++k) {
                rays[6 * i + k] = of[k];
                rays[6 * i + 3 + k] = df[k];
            }
            break;
        }
        total += a + 1;
        if (a == max_attempts) failed |= 1;
    }
    return failed ? -1 : total;
}
