/*
 * CPU oracle for the per-frame distance-map pipeline of "Real Time Collision
 * Avoidance with GPU-Computed Distance Maps" (arXiv 2407.02363).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this file; only the tests, the smoke check and the bench's CPU-baseline leg do.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Plain, slow, obviously correct code:
 *   - occupancy insertion of points and of FK-placed link voxels (Alg. 2, lines 5-7;
 *     Sec. III-A), in fp32 with the operation order spelled out below, because the
 *     floating-point voxelisation decides an integer voxel index and both sides must
 *     take that decision in the same precision;
 *   - the exact EDT (Sec. III-C), as the separable row / column / stack procedure
 *     of Alg. 1 with bands m1 = m2 = m3 = 1, in int64 arithmetic;
 *   - the EDT by its definition (min over all occupied voxels), for pinning;
 *   - the sphere query of Eq. (dist) / Alg. 3 lines 3-4 (ExtractClosestObstaclePose).
 *
 * Grid layout: uint8 occ[z][y][x], linear index x + X*(y + Y*z); any nonzero byte
 * is an occupied voxel.  Squared distances are in voxel units.  An empty map gives
 * sqdist = INT32_MAX and idx = -1 everywhere.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see oracle/build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NONE_SITE (-1)

/* ------------------------------------------------------------------------------ */
/* Voxelisation: v = floor((p - origin) / vs) in fp32, inside iff 0 <= v < n.       */
/* Points exactly on the upper face and NaN points fall outside.                     */
/* ------------------------------------------------------------------------------ */
static int voxel_coord(float p, float o, float vs, int n, int *v)
{
    float d = p - o;        /* one IEEE round-to-nearest subtraction */
    float q = d / vs;       /* one IEEE round-to-nearest division    */
    float f = floorf(q);
    if (!(f >= 0.0f) || !(f < (float)n)) return 0;
    *v = (int)f;
    return 1;
}

/* Rigid transform w = R p + t with the row sums taken left to right, no FMA:
 * w_a = ((R_a0 p_x + R_a1 p_y) + R_a2 p_z) + t_a.  T is 3x4 row-major (R | t). */
static void transform(const float *T, const float *p, float *w)
{
    for (int a = 0; a < 3; a++) {
        float s = T[4 * a + 0] * p[0];
        float u = T[4 * a + 1] * p[1];
        s = s + u;
        u = T[4 * a + 2] * p[2];
        s = s + u;
        w[a] = s + T[4 * a + 3];
    }
}

/* Insert(Point_Cloud), Alg. 2 line 7, with the robot-voxel removal of Sec. III-A:
 * every point (optionally moved by T_world_sensor) marks its voxel in env; a point
 * whose voxel is occupied in the self map is dropped when filter_self is set.
 * Returns the number of points written. */
int64_t oracle_insert_points(uint8_t *env, const uint8_t *self, int X, int Y, int Z,
                             float vs, const float *origin, const float *xyz, int64_t n,
                             const float *T, int filter_self)
{
    int64_t written = 0;
    for (int64_t i = 0; i < n; i++) {
        float p[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
        float w[3];
        if (T) transform(T, p, w);
        else { w[0] = p[0]; w[1] = p[1]; w[2] = p[2]; }
        int vx, vy, vz;
        if (!voxel_coord(w[0], origin[0], vs, X, &vx)) continue;
        if (!voxel_coord(w[1], origin[1], vs, Y, &vy)) continue;
        if (!voxel_coord(w[2], origin[2], vs, Z, &vz)) continue;
        int64_t id = (int64_t)vx + (int64_t)X * ((int64_t)vy + (int64_t)Y * vz);
        if (filter_self && self && self[id]) continue;
        env[id] = 1;
        written++;
    }
    return written;
}

/* UpdateLinks + Insert(O_Lk), Alg. 2 lines 5-6 (Sec. III-A, III-E): link k's offline
 * voxel model (points pts[offs[k] .. offs[k+1]) in the link frame) is moved by its fp32
 * pose poses[12k .. 12k+12) and marked in the self map, for links whose bit is set in
 * link_mask.  Returns the number of link points that landed inside the grid. */
int64_t oracle_insert_links(uint8_t *self, int X, int Y, int Z, float vs, const float *origin,
                            int n_links, const float *pts, const int64_t *offs,
                            const float *poses, uint32_t link_mask)
{
    int64_t written = 0;
    for (int k = 0; k < n_links; k++) {
        if (!((link_mask >> k) & 1u)) continue;
        for (int64_t i = offs[k]; i < offs[k + 1]; i++) {
            float w[3];
            transform(poses + 12 * k, pts + 3 * i, w);
            int vx, vy, vz;
            if (!voxel_coord(w[0], origin[0], vs, X, &vx)) continue;
            if (!voxel_coord(w[1], origin[1], vs, Y, &vy)) continue;
            if (!voxel_coord(w[2], origin[2], vs, Z, &vz)) continue;
            self[(int64_t)vx + (int64_t)X * ((int64_t)vy + (int64_t)Y * vz)] = 1;
            written++;
        }
    }
    return written;
}

/* ------------------------------------------------------------------------------ */
/* Exact EDT, separable form of Alg. 1 (Sec. III-C) with m1 = m2 = m3 = 1.            */
/* ------------------------------------------------------------------------------ */

/* ComputeProximateSite + QueryNearestSite on one line of n voxels (Steps 2-3, and
 * Step 4 along the stacking axis).  Site s exists iff has[s]; its parabola is
 * f[s] + (j - s)^2.  Sites are swept in increasing order keeping a stack of
 * potentially proximate sites; the top b is popped while it is dominated by the new
 * site c and the site a below it, i.e. while the point where c overtakes b does not
 * come after the point where b overtakes a:
 *     (h_c - h_b)(b - a) <= (h_b - h_a)(c - b),   h_s = f[s] + s^2.
 * Then each voxel j walks the stack upward while the next proximate site is strictly
 * closer.  arg[j] = nearest site (NONE_SITE if the line has none), val[j] its value. */
static void envelope_line(int n, const int64_t *f, const uint8_t *has, int *stk,
                          int32_t *arg, int64_t *val)
{
    int k = 0;
    for (int c = 0; c < n; c++) {
        if (!has[c]) continue;
        int64_t hc = f[c] + (int64_t)c * c;
        while (k >= 2) {
            int a = stk[k - 2], b = stk[k - 1];
            int64_t ha = f[a] + (int64_t)a * a;
            int64_t hb = f[b] + (int64_t)b * b;
            if ((hc - hb) * (int64_t)(b - a) <= (hb - ha) * (int64_t)(c - b)) k--;
            else break;
        }
        stk[k++] = c;
    }
    int p = 0;
    for (int j = 0; j < n; j++) {
        if (k == 0) { arg[j] = NONE_SITE; val[j] = 0; continue; }
        for (;;) {
            if (p + 1 >= k) break;
            int64_t d0 = (int64_t)(j - stk[p]), d1 = (int64_t)(j - stk[p + 1]);
            int64_t v0 = f[stk[p]] + d0 * d0, v1 = f[stk[p + 1]] + d1 * d1;
            if (v1 < v0) p++; else break;
        }
        int64_t d = (int64_t)(j - stk[p]);
        arg[j] = stk[p];
        val[j] = f[stk[p]] + d * d;
    }
}

void oracle_edt(const uint8_t *occ, int X, int Y, int Z, int32_t *sqdist, int32_t *idx,
                int nthreads)
{
    const int64_t N = (int64_t)X * Y * Z;
    int32_t *xs = (int32_t *)malloc(sizeof(int32_t) * N);   /* Step 1: nearest x in row  */
    int32_t *ys = (int32_t *)malloc(sizeof(int32_t) * N);   /* Step 3: 2-D site's y       */
    int64_t *g2 = (int64_t *)malloc(sizeof(int64_t) * N);   /* Step 3: squared 2-D dist   */
    uint8_t *slice_has = (uint8_t *)calloc((size_t)Z, 1);
    if (nthreads < 1) nthreads = 1;

    /* Step 1 (BandSweep + PropagateAcrossBand with m1 = 1): for voxel (i, j, k), the
     * nearest site among the sites of row j of slice k; two sweeps per row. */
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int64_t r = 0; r < (int64_t)Y * Z; r++) {
        const uint8_t *row = occ + r * X;
        int32_t *out = xs + r * X;
        int last = NONE_SITE;
        for (int i = 0; i < X; i++) {
            if (row[i]) last = i;
            out[i] = last;
        }
        last = NONE_SITE;
        for (int i = X - 1; i >= 0; i--) {
            if (row[i]) last = i;
            if (last != NONE_SITE && (out[i] == NONE_SITE || (last - i) < (i - out[i])))
                out[i] = last;
        }
    }

    /* Steps 2-3 in every slice k and column i, along y. */
#pragma omp parallel num_threads(nthreads)
    {
        int64_t *f = (int64_t *)malloc(sizeof(int64_t) * Y);
        uint8_t *has = (uint8_t *)malloc((size_t)Y);
        int *stk = (int *)malloc(sizeof(int) * Y);
        int32_t *arg = (int32_t *)malloc(sizeof(int32_t) * Y);
        int64_t *val = (int64_t *)malloc(sizeof(int64_t) * Y);
#pragma omp for schedule(static)
        for (int64_t c = 0; c < (int64_t)X * Z; c++) {
            int i = (int)(c % X);
            int64_t k = c / X;
            int any = 0;
            for (int j = 0; j < Y; j++) {
                int32_t s = xs[i + (int64_t)X * (j + (int64_t)Y * k)];
                has[j] = s != NONE_SITE;
                f[j] = has[j] ? (int64_t)(i - s) * (i - s) : 0;
                any |= has[j];
            }
            envelope_line(Y, f, has, stk, arg, val);
            for (int j = 0; j < Y; j++) {
                int64_t id = i + (int64_t)X * (j + (int64_t)Y * k);
                ys[id] = arg[j];
                g2[id] = val[j];
            }
            if (any) slice_has[k] = 1;   /* every column of a non-empty slice agrees */
        }
        free(f); free(has); free(stk); free(arg); free(val);
    }

    /* Step 4: Steps 2-3 repeated along z on the stack of 2-D results. */
#pragma omp parallel num_threads(nthreads)
    {
        int64_t *f = (int64_t *)malloc(sizeof(int64_t) * Z);
        int *stk = (int *)malloc(sizeof(int) * Z);
        int32_t *arg = (int32_t *)malloc(sizeof(int32_t) * Z);
        int64_t *val = (int64_t *)malloc(sizeof(int64_t) * Z);
#pragma omp for schedule(static)
        for (int64_t c = 0; c < (int64_t)X * Y; c++) {
            for (int k = 0; k < Z; k++) f[k] = slice_has[k] ? g2[c + (int64_t)X * Y * k] : 0;
            envelope_line(Z, f, slice_has, stk, arg, val);
            int i = (int)(c % X);
            int j0 = (int)(c / X);
            for (int k = 0; k < Z; k++) {
                int64_t id = c + (int64_t)X * Y * k;
                if (arg[k] == NONE_SITE) { sqdist[id] = INT32_MAX; idx[id] = -1; continue; }
                int64_t src = c + (int64_t)X * Y * arg[k];          /* voxel (i, j0, z*)  */
                int32_t ystar = ys[src];
                int32_t xstar = xs[i + (int64_t)X * (ystar + (int64_t)Y * arg[k])];
                sqdist[id] = (int32_t)val[k];
                idx[id] = (int32_t)(xstar + (int64_t)X * (ystar + (int64_t)Y * arg[k]));
                (void)j0;
            }
        }
        free(f); free(stk); free(arg); free(val);
    }
    free(xs); free(ys); free(g2); free(slice_has);
}

/* The EDT by its definition: for each queried voxel, the minimum over every occupied
 * voxel s of |v - s|^2 (ties keep the lowest linear index). */
void oracle_edt_brute(const uint8_t *occ, int X, int Y, int Z, const int64_t *query,
                      int64_t nq, int32_t *sqdist, int32_t *idx, int nthreads)
{
    const int64_t N = (int64_t)X * Y * Z;
    int64_t ns = 0;
    for (int64_t i = 0; i < N; i++) ns += occ[i] != 0;
    int32_t *sx = (int32_t *)malloc(sizeof(int32_t) * (ns + 1));
    int32_t *sy = (int32_t *)malloc(sizeof(int32_t) * (ns + 1));
    int32_t *sz = (int32_t *)malloc(sizeof(int32_t) * (ns + 1));
    int64_t w = 0;
    for (int64_t i = 0; i < N; i++) {
        if (!occ[i]) continue;
        sx[w] = (int32_t)(i % X);
        sy[w] = (int32_t)((i / X) % Y);
        sz[w] = (int32_t)(i / ((int64_t)X * Y));
        w++;
    }
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 64)
    for (int64_t q = 0; q < nq; q++) {
        int64_t v = query[q];
        int64_t x = v % X, y = (v / X) % Y, z = v / ((int64_t)X * Y);
        int64_t best = INT64_MAX, bi = -1;
        for (int64_t s = 0; s < ns; s++) {
            int64_t dx = x - sx[s], dy = y - sy[s], dz = z - sz[s];
            int64_t d = dx * dx + dy * dy + dz * dz;
            if (d < best) { best = d; bi = sx[s] + (int64_t)X * (sy[s] + (int64_t)Y * sz[s]); }
        }
        sqdist[q] = bi < 0 ? INT32_MAX : (int32_t)best;
        idx[q] = (int32_t)bi;
    }
    free(sx); free(sy); free(sz);
}

/* ------------------------------------------------------------------------------ */
/* ExtractClosestObstaclePose + Eq. (dist) (Alg. 2 line 10; Alg. 3 lines 3-4).       */
/* ------------------------------------------------------------------------------ */
typedef struct {
    int32_t sqdist;      /* squared voxel distance at the centre's voxel              */
    int32_t idx;         /* linear index of the nearest occupied voxel, -1 if none    */
    float dist;          /* metres: vs * sqrt(sqdist)                                 */
    float clearance;     /* dist - radius                                             */
    float nearest[3];    /* world centre of the nearest occupied voxel                */
    int32_t status;      /* 0 ok, 1 centre outside the grid, 2 map empty              */
} oracle_sphere;

void oracle_query(const int32_t *sqdist, const int32_t *idx, int X, int Y, int Z, float vs,
                  const float *origin, const float *centres, const float *radii, int m,
                  oracle_sphere *out)
{
    for (int i = 0; i < m; i++) {
        oracle_sphere r;
        int v[3];
        int dims[3] = {X, Y, Z};
        int inside = 1;
        for (int a = 0; a < 3; a++)
            inside &= voxel_coord(centres[3 * i + a], origin[a], vs, dims[a], &v[a]);
        if (!inside) {
            r.sqdist = -1; r.idx = -1; r.dist = NAN; r.clearance = NAN;
            r.nearest[0] = r.nearest[1] = r.nearest[2] = NAN; r.status = 1;
            out[i] = r;
            continue;
        }
        int64_t id = v[0] + (int64_t)X * (v[1] + (int64_t)Y * v[2]);
        r.sqdist = sqdist[id];
        r.idx = idx[id];
        if (r.idx < 0) {
            r.dist = INFINITY; r.clearance = INFINITY;
            r.nearest[0] = r.nearest[1] = r.nearest[2] = NAN; r.status = 2;
            out[i] = r;
            continue;
        }
        float fd = (float)r.sqdist;              /* exact: sqdist < 2^24 */
        float sq = sqrtf(fd);                    /* IEEE correctly rounded */
        r.dist = vs * sq;
        r.clearance = r.dist - radii[i];
        int64_t j = r.idx;
        int nv[3] = {(int)(j % X), (int)((j / X) % Y), (int)(j / ((int64_t)X * Y))};
        for (int a = 0; a < 3; a++) {
            float c = (float)nv[a] + 0.5f;       /* exact */
            float s = c * vs;
            r.nearest[a] = origin[a] + s;
        }
        r.status = 0;
        out[i] = r;
    }
}
