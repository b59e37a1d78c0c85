/*
 * Oracle for the cell-mechanics step: plain, slow, FP64, CPU only.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header or constant with the CUDA
 * library.
 *
 * What it computes (the "update velocity" region of the agent-based
 * simulation analysed in Sec. 5.4 of the paper: a loop over all cells that
 * updates each cell's velocity from its neighbouring cells, found through the
 * mechanics voxel grid of Listing 4):
 *
 *   1. Binning.  Each cell gets the voxel index
 *        i_d = clamp(floor((x_d - lo_d) * inv_h), 0, n_d - 1),  inv_h = 1/h,
 *      key = i_x + n_x * (i_y + n_y * i_z), and the cells are put in voxel
 *      order by a stable counting sort of the keys listed in ascending cell
 *      index, i.e. within a voxel cells stay in ascending index order.
 *   2. Velocity.  For each cell i, every cell j != i in the 27 voxels around
 *      i's voxel with d = |x_i - x_j| > 0 and S = R_i + R_j contributes
 *        c_r = sqrt(ccr_i ccr_j) (1 - d/S)^2          if d < S   (repulsion)
 *        c_a = sqrt(cca_i cca_j) (1 - d/(A S))^2      if d < A S (adhesion)
 *        v_i += (c_r - c_a) (x_i - x_j) / d.
 *      Neighbour voxels are visited in lexicographic (dz, dy, dx) order,
 *      cells inside a voxel in sorted order, and the sum is taken in FP64 in
 *      that order, so the result does not depend on the thread count.
 *   3. Integration by two-step Adams-Bashforth:
 *        x_{n+1} = x_n + dt (1.5 v_n - 0.5 v_{n-1}),  v_{-1} = 0.
 *
 * The paper states none of these formulas (it analyses PhysiCell's
 * implementation); the force law, the AB2 integrator and the binning are the
 * statement of the problem this library solves, restated here.  Readings of
 * unstated details (clamping of cells outside the domain, the rounding of the
 * voxel index, strict cutoff comparisons, order inside a voxel) are listed in
 * the design notes of the repository.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math: all
 * arithmetic is IEEE double with round-to-nearest and no FMA contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double lo[3];
    double h;
    double inv_h;
    int32_t n[3];
} grid_t;

static void grid_init(grid_t* g, const double lo[3], double h, const int32_t n[3]) {
    for (int d = 0; d < 3; ++d) { g->lo[d] = lo[d]; g->n[d] = n[d]; }
    g->h = h;
    g->inv_h = 1.0 / h;
}

/* Voxel index along one axis, FP64 (step 1). */
static int32_t axis_index_f64(double x, double lo, double inv_h, int32_t n) {
    double t = (x - lo) * inv_h;
    double f = floor(t);
    if (!(f >= 0.0)) return 0;              /* below the domain (or NaN): first voxel */
    if (f >= (double)(n - 1)) return n - 1; /* above the domain: last voxel */
    return (int32_t)f;
}

/* Same in FP32, for positions held as FP32 (compensated-position mode): the
 * index decision is taken in the precision of the positions themselves. */
static int32_t axis_index_f32(float x, float lo, float inv_h, int32_t n) {
    float t = (x - lo) * inv_h;
    float f = floorf(t);
    if (!(f >= 0.0f)) return 0;
    if (f >= (float)(n - 1)) return n - 1;
    return (int32_t)f;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Step 1a: voxel keys from FP64 positions (xyz interleaved, 3n doubles). */
void oracle_keys(int64_t n, const double* xyz, const double lo[3], double h,
                 const int32_t dims[3], uint32_t* key) {
    grid_t g;
    grid_init(&g, lo, h, dims);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int32_t ix = axis_index_f64(xyz[3 * i + 0], g.lo[0], g.inv_h, g.n[0]);
        int32_t iy = axis_index_f64(xyz[3 * i + 1], g.lo[1], g.inv_h, g.n[1]);
        int32_t iz = axis_index_f64(xyz[3 * i + 2], g.lo[2], g.inv_h, g.n[2]);
        key[i] = (uint32_t)ix + (uint32_t)g.n[0] * ((uint32_t)iy + (uint32_t)g.n[1] * (uint32_t)iz);
    }
}

/* Step 1a for FP32 positions: lo and inv_h are first rounded to FP32. */
void oracle_keys_f32(int64_t n, const float* xyz, const double lo[3], double h,
                     const int32_t dims[3], uint32_t* key) {
    float lof[3] = {(float)lo[0], (float)lo[1], (float)lo[2]};
    float invf = (float)(1.0 / h);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int32_t ix = axis_index_f32(xyz[3 * i + 0], lof[0], invf, dims[0]);
        int32_t iy = axis_index_f32(xyz[3 * i + 1], lof[1], invf, dims[1]);
        int32_t iz = axis_index_f32(xyz[3 * i + 2], lof[2], invf, dims[2]);
        key[i] = (uint32_t)ix + (uint32_t)dims[0] * ((uint32_t)iy + (uint32_t)dims[1] * (uint32_t)iz);
    }
}

/* Step 1b: stable counting sort.  count[V], start[V+1] (exclusive prefix sum
 * of count), order[n]: order[p] = index of the cell at sorted position p.
 * Sequential on purpose: it is the definition. */
void oracle_counting_sort(int64_t n, const uint32_t* key, int64_t V,
                          uint32_t* count, uint32_t* start, int64_t* order) {
    memset(count, 0, (size_t)V * sizeof(uint32_t));
    for (int64_t i = 0; i < n; ++i) count[key[i]] += 1;
    uint64_t run = 0;
    for (int64_t v = 0; v < V; ++v) { start[v] = (uint32_t)run; run += count[v]; }
    start[V] = (uint32_t)run;
    uint32_t* fill = (uint32_t*)malloc((size_t)(V > 0 ? V : 1) * sizeof(uint32_t));
    memcpy(fill, start, (size_t)V * sizeof(uint32_t));
    for (int64_t i = 0; i < n; ++i) order[fill[key[i]]++] = i;
    free(fill);
}

/* Pair term of step 2 for cells i, j; adds to acc[3].  Returns 1 if the pair
 * interacts (0 < d < A S). */
static int pair_term(const double* xi, const double* xj, double Ri, double Rj,
                     double ccri, double ccrj, double ccai, double ccaj,
                     double A, double acc[3]) {
    double dx = xi[0] - xj[0];
    double dy = xi[1] - xj[1];
    double dz = xi[2] - xj[2];
    double d2 = dx * dx + dy * dy + dz * dz;
    double d = sqrt(d2);
    if (!(d > 0.0)) return 0;
    double S = Ri + Rj;
    double AS = A * S;
    if (!(d < AS)) return 0;
    double c = 0.0;
    if (d < S) {
        double t = 1.0 - d / S;
        c = sqrt(ccri * ccrj) * (t * t);
    }
    double ta = 1.0 - d / AS;
    c = c - sqrt(ccai * ccaj) * (ta * ta);
    double s = c / d;
    acc[0] += s * dx;
    acc[1] += s * dy;
    acc[2] += s * dz;
    return 1;
}

typedef struct {
    grid_t g;
    int64_t V;
    uint32_t* key;
    uint32_t* count;
    uint32_t* start;
    int64_t* order;
} bins_t;

static int bins_build(bins_t* b, int64_t n, const double* xyz, const double lo[3],
                      double h, const int32_t dims[3]) {
    grid_init(&b->g, lo, h, dims);
    b->V = (int64_t)dims[0] * dims[1] * dims[2];
    b->key = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
    b->count = (uint32_t*)malloc((size_t)b->V * sizeof(uint32_t));
    b->start = (uint32_t*)malloc((size_t)(b->V + 1) * sizeof(uint32_t));
    b->order = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!b->key || !b->count || !b->start || !b->order) return -1;
    oracle_keys(n, xyz, lo, h, dims, b->key);
    oracle_counting_sort(n, b->key, b->V, b->count, b->start, b->order);
    return 0;
}

static void bins_free(bins_t* b) {
    free(b->key); free(b->count); free(b->start); free(b->order);
}

/* Velocity of one cell by the binned neighbour search of step 2. */
static void velocity_one(int64_t i, const bins_t* b, const double* xyz, const double* R,
                         const double* ccr, const double* cca, double A, double out[3]) {
    const int32_t* n = b->g.n;
    uint32_t k = b->key[i];
    int32_t ix = (int32_t)(k % (uint32_t)n[0]);
    int32_t iy = (int32_t)((k / (uint32_t)n[0]) % (uint32_t)n[1]);
    int32_t iz = (int32_t)(k / ((uint32_t)n[0] * (uint32_t)n[1]));
    double acc[3] = {0.0, 0.0, 0.0};
    for (int dz = -1; dz <= 1; ++dz) {
        int32_t jz = iz + dz;
        if (jz < 0 || jz >= n[2]) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int32_t jy = iy + dy;
            if (jy < 0 || jy >= n[1]) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                int32_t jx = ix + dx;
                if (jx < 0 || jx >= n[0]) continue;
                uint32_t vk = (uint32_t)jx + (uint32_t)n[0] * ((uint32_t)jy + (uint32_t)n[1] * (uint32_t)jz);
                for (uint32_t q = b->start[vk]; q < b->start[vk + 1]; ++q) {
                    int64_t j = b->order[q];
                    if (j == i) continue;
                    pair_term(&xyz[3 * i], &xyz[3 * j], R[i], R[j], ccr[i], ccr[j],
                              cca[i], cca[j], A, acc);
                }
            }
        }
    }
    out[0] = acc[0]; out[1] = acc[1]; out[2] = acc[2];
}

/* Step 2 for all cells (binned).  v: 3n doubles, caller's cell order. */
int oracle_velocities(int64_t n, const double* xyz, const double* R, const double* ccr,
                      const double* cca, double A, const double lo[3], double h,
                      const int32_t dims[3], double* v) {
    bins_t b;
    if (bins_build(&b, n, xyz, lo, h, dims) != 0) { bins_free(&b); return -1; }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) velocity_one(i, &b, xyz, R, ccr, cca, A, &v[3 * i]);
    bins_free(&b);
    return 0;
}

/* Step 2 for the listed cells only (full binning, velocities of idx[] only). */
int oracle_velocities_subset(int64_t n, const double* xyz, const double* R, const double* ccr,
                             const double* cca, double A, const double lo[3], double h,
                             const int32_t dims[3], int64_t m, const int64_t* idx, double* v) {
    bins_t b;
    if (bins_build(&b, n, xyz, lo, h, dims) != 0) { bins_free(&b); return -1; }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < m; ++k) velocity_one(idx[k], &b, xyz, R, ccr, cca, A, &v[3 * k]);
    bins_free(&b);
    return 0;
}

/* Step 2 by all pairs, O(n^2): no binning at all.  Sum over j in ascending
 * index order. */
void oracle_velocities_allpairs(int64_t n, const double* xyz, const double* R, const double* ccr,
                                const double* cca, double A, double* v) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            pair_term(&xyz[3 * i], &xyz[3 * j], R[i], R[j], ccr[i], ccr[j], cca[i], cca[j], A, acc);
        }
        v[3 * i] = acc[0]; v[3 * i + 1] = acc[1]; v[3 * i + 2] = acc[2];
    }
}

/* Interacting pairs (i < j, 0 < d < A S) found through the bins.  Writes up
 * to max_pairs (i, j) pairs into pairs[2*k], pairs[2*k+1]; returns the total
 * count (sequential, so the list order is deterministic). */
int64_t oracle_pairs(int64_t n, const double* xyz, const double* R, double A,
                     const double lo[3], double h, const int32_t dims[3],
                     int64_t max_pairs, int64_t* pairs) {
    bins_t b;
    if (bins_build(&b, n, xyz, lo, h, dims) != 0) { bins_free(&b); return -1; }
    const int32_t* nd = b.g.n;
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t k = b.key[i];
        int32_t ix = (int32_t)(k % (uint32_t)nd[0]);
        int32_t iy = (int32_t)((k / (uint32_t)nd[0]) % (uint32_t)nd[1]);
        int32_t iz = (int32_t)(k / ((uint32_t)nd[0] * (uint32_t)nd[1]));
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int32_t jx = ix + dx, jy = iy + dy, jz = iz + dz;
                    if (jx < 0 || jx >= nd[0] || jy < 0 || jy >= nd[1] || jz < 0 || jz >= nd[2]) continue;
                    uint32_t vk = (uint32_t)jx + (uint32_t)nd[0] * ((uint32_t)jy + (uint32_t)nd[1] * (uint32_t)jz);
                    for (uint32_t q = b.start[vk]; q < b.start[vk + 1]; ++q) {
                        int64_t j = b.order[q];
                        if (j <= i) continue;
                        double ddx = xyz[3 * i] - xyz[3 * j], ddy = xyz[3 * i + 1] - xyz[3 * j + 1],
                               ddz = xyz[3 * i + 2] - xyz[3 * j + 2];
                        double d = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
                        if (d > 0.0 && d < A * (R[i] + R[j])) {
                            if (cnt < max_pairs) { pairs[2 * cnt] = i; pairs[2 * cnt + 1] = j; }
                            ++cnt;
                        }
                    }
                }
    }
    bins_free(&b);
    return cnt;
}

/* Same pair set by all pairs (no bins). */
int64_t oracle_pairs_allpairs(int64_t n, const double* xyz, const double* R, double A,
                              int64_t max_pairs, int64_t* pairs) {
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double ddx = xyz[3 * i] - xyz[3 * j], ddy = xyz[3 * i + 1] - xyz[3 * j + 1],
                   ddz = xyz[3 * i + 2] - xyz[3 * j + 2];
            double d = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
            if (d > 0.0 && d < A * (R[i] + R[j])) {
                if (cnt < max_pairs) { pairs[2 * cnt] = i; pairs[2 * cnt + 1] = j; }
                ++cnt;
            }
        }
    return cnt;
}

/* Step 3: x += dt (1.5 v - 0.5 vprev), then vprev <- v. */
void oracle_ab2(int64_t n, double* xyz, const double* v, double* vprev, double dt) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < 3 * n; ++k) {
        xyz[k] = xyz[k] + dt * (1.5 * v[k] - 0.5 * vprev[k]);
        vprev[k] = v[k];
    }
}

/* Full steps 1-3, `steps` times.  xyz and vprev are updated in place; v (3n)
 * receives the velocity of the last step (computed from the positions at the
 * start of that step).  Returns 0, or -1 on allocation failure. */
int oracle_run(int64_t n, double* xyz, double* vprev, const double* R, const double* ccr,
               const double* cca, double A, const double lo[3], double h,
               const int32_t dims[3], double dt, int64_t steps, double* v) {
    for (int64_t s = 0; s < steps; ++s) {
        if (oracle_velocities(n, xyz, R, ccr, cca, A, lo, h, dims, v) != 0) return -1;
        oracle_ab2(n, xyz, v, vprev, dt);
    }
    return 0;
}

/*
 * Velocity variants (the "update velocity" region with two PhysiCell-style
 * extensions the paper names the system for but does not state; the
 * statement is ours):
 *
 *   Per-type adhesion affinity.  Every cell carries a type t in [0, T); a
 *   symmetric T x T matrix a (entries >= 0) scales the adhesion coefficient
 *   of a pair:  c_a = (a[t_i][t_j] * sqrt(cca_i cca_j)) (1 - d/(A S))^2,
 *   the product taken in that order.  All entries 1 is the base law.
 *
 *   Domain walls.  Each enabled face of the box [wlo, whi] (bit f of `mask`
 *   for the faces -x, +x, -y, +y, -z, +z, in that order) pushes a cell
 *   inward when the cell overlaps it: with d_w the distance of the centre
 *   from the face plane, measured inward (x_d - wlo_d for a low face,
 *   whi_d - x_d for a high face), and n the inward unit normal,
 *       t = 1 - d_w / R_i  if 0 < d_w < R_i,   t = 1  if d_w <= 0,
 *       v_i += c_w t^2 n   (nothing if d_w >= R_i),
 *   added after the pair terms, face by face in the order above.
 */
typedef struct {
    int32_t ntypes;
    const int32_t* type;  /* per cell, in [0, ntypes) */
    const double* aff;    /* ntypes x ntypes, row-major, symmetric */
    int32_t mask;         /* enabled faces */
    double wlo[3], whi[3];
    double cw;            /* wall coefficient (um/min) */
} variant_t;

/* Pair term with the affinity factor (step 2 of the variant). */
static void pair_term_aff(const double* xi, const double* xj, double Ri, double Rj, double ccri, double ccrj,
                          double ccai, double ccaj, double aij, double A, double acc[3]) {
    double dx = xi[0] - xj[0];
    double dy = xi[1] - xj[1];
    double dz = xi[2] - xj[2];
    double d2 = dx * dx + dy * dy + dz * dz;
    double d = sqrt(d2);
    if (!(d > 0.0)) return;
    double S = Ri + Rj;
    double AS = A * S;
    if (!(d < AS)) return;
    double c = 0.0;
    if (d < S) {
        double t = 1.0 - d / S;
        c = sqrt(ccri * ccrj) * (t * t);
    }
    double ta = 1.0 - d / AS;
    c = c - (aij * sqrt(ccai * ccaj)) * (ta * ta);
    double s = c / d;
    acc[0] += s * dx;
    acc[1] += s * dy;
    acc[2] += s * dz;
}

/* Wall terms of one cell, added to acc in face order. */
static void wall_terms(const double* x, double Ri, const variant_t* w, double acc[3]) {
    for (int f = 0; f < 6; ++f) {
        if (!(w->mask & (1 << f))) continue;
        int axis = f / 2;
        int high = f % 2;
        double dw = high ? w->whi[axis] - x[axis] : x[axis] - w->wlo[axis];
        if (!(dw < Ri)) continue;
        double t = dw > 0.0 ? 1.0 - dw / Ri : 1.0;
        double push = w->cw * (t * t);
        acc[axis] += high ? -push : push;
    }
}

static double affinity(const variant_t* w, int64_t i, int64_t j) {
    return w->aff[(int64_t)w->type[i] * w->ntypes + w->type[j]];
}

static void velocity_one_ext(int64_t i, const bins_t* b, const double* xyz, const double* R, const double* ccr,
                             const double* cca, double A, const variant_t* w, double out[3]) {
    const int32_t* n = b->g.n;
    uint32_t k = b->key[i];
    int32_t ix = (int32_t)(k % (uint32_t)n[0]);
    int32_t iy = (int32_t)((k / (uint32_t)n[0]) % (uint32_t)n[1]);
    int32_t iz = (int32_t)(k / ((uint32_t)n[0] * (uint32_t)n[1]));
    double acc[3] = {0.0, 0.0, 0.0};
    for (int dz = -1; dz <= 1; ++dz) {
        int32_t jz = iz + dz;
        if (jz < 0 || jz >= n[2]) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int32_t jy = iy + dy;
            if (jy < 0 || jy >= n[1]) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                int32_t jx = ix + dx;
                if (jx < 0 || jx >= n[0]) continue;
                uint32_t vk = (uint32_t)jx + (uint32_t)n[0] * ((uint32_t)jy + (uint32_t)n[1] * (uint32_t)jz);
                for (uint32_t q = b->start[vk]; q < b->start[vk + 1]; ++q) {
                    int64_t j = b->order[q];
                    if (j == i) continue;
                    pair_term_aff(&xyz[3 * i], &xyz[3 * j], R[i], R[j], ccr[i], ccr[j], cca[i], cca[j],
                                  affinity(w, i, j), A, acc);
                }
            }
        }
    }
    wall_terms(&xyz[3 * i], R[i], w, acc);
    out[0] = acc[0]; out[1] = acc[1]; out[2] = acc[2];
}

static void variant_init(variant_t* w, int32_t ntypes, const int32_t* type, const double* aff, int32_t mask,
                         const double wlo[3], const double whi[3], double cw) {
    w->ntypes = ntypes;
    w->type = type;
    w->aff = aff;
    w->mask = mask;
    for (int d = 0; d < 3; ++d) { w->wlo[d] = wlo[d]; w->whi[d] = whi[d]; }
    w->cw = cw;
}

/* Step 2 with the variants, binned. */
int oracle_velocities_ext(int64_t n, const double* xyz, const double* R, const double* ccr, const double* cca,
                          double A, const double lo[3], double h, const int32_t dims[3], int32_t ntypes,
                          const int32_t* type, const double* aff, int32_t mask, const double wlo[3],
                          const double whi[3], double cw, double* v) {
    variant_t w;
    variant_init(&w, ntypes, type, aff, mask, wlo, whi, cw);
    bins_t b;
    if (bins_build(&b, n, xyz, lo, h, dims) != 0) { bins_free(&b); return -1; }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) velocity_one_ext(i, &b, xyz, R, ccr, cca, A, &w, &v[3 * i]);
    bins_free(&b);
    return 0;
}

/* Step 2 with the variants by all pairs (j ascending), no binning. */
void oracle_velocities_allpairs_ext(int64_t n, const double* xyz, const double* R, const double* ccr,
                                    const double* cca, double A, int32_t ntypes, const int32_t* type,
                                    const double* aff, int32_t mask, const double wlo[3], const double whi[3],
                                    double cw, double* v) {
    variant_t w;
    variant_init(&w, ntypes, type, aff, mask, wlo, whi, cw);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            pair_term_aff(&xyz[3 * i], &xyz[3 * j], R[i], R[j], ccr[i], ccr[j], cca[i], cca[j],
                          affinity(&w, i, j), A, acc);
        }
        wall_terms(&xyz[3 * i], R[i], &w, acc);
        v[3 * i] = acc[0]; v[3 * i + 1] = acc[1]; v[3 * i + 2] = acc[2];
    }
}

/* Full steps 1-3 with the variants (as oracle_run). */
int oracle_run_ext(int64_t n, double* xyz, double* vprev, const double* R, const double* ccr, const double* cca,
                   double A, const double lo[3], double h, const int32_t dims[3], int32_t ntypes,
                   const int32_t* type, const double* aff, int32_t mask, const double wlo[3], const double whi[3],
                   double cw, double dt, int64_t steps, double* v) {
    for (int64_t s = 0; s < steps; ++s) {
        if (oracle_velocities_ext(n, xyz, R, ccr, cca, A, lo, h, dims, ntypes, type, aff, mask, wlo, whi, cw,
                                  v) != 0)
            return -1;
        oracle_ab2(n, xyz, v, vprev, dt);
    }
    return 0;
}
