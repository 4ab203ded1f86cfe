/*
 * Driver that runs the C oracle under AddressSanitizer and UndefinedBehaviorSanitizer
 * (built and run by tests/test_oracle_sanitizers.py): every entry point on small grids,
 * ragged and one-dimensional shapes, empty and full maps, points and spheres outside
 * the grid or NaN, with the EDT checked against the brute-force definition.  Any
 * out-of-bounds access, leak or undefined operation aborts the run; a wrong distance
 * makes it exit 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t sqdist, idx;
    float dist, clearance, nearest[3];
    int32_t status;
} sphere_out;

int64_t oracle_insert_points(uint8_t *env, const uint8_t *self, int X, int Y, int Z, float vs,
                             const float *origin, const float *xyz, int64_t n, const float *T,
                             int filter_self);
int64_t oracle_insert_links(uint8_t *self, int X, int Y, int Z, float vs, const float *origin,
                            int n_links, const float *pts, const int64_t *offs, const float *poses,
                            uint32_t link_mask);
void oracle_edt(const uint8_t *occ, int X, int Y, int Z, int32_t *sqdist, int32_t *idx, int nthreads);
void oracle_edt_brute(const uint8_t *occ, int X, int Y, int Z, const int64_t *query, int64_t nq,
                      int32_t *sqdist, int32_t *idx, int nthreads);
void oracle_query(const int32_t *sqdist, const int32_t *idx, int X, int Y, int Z, float vs,
                  const float *origin, const float *centres, const float *radii, int m, sphere_out *out);

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static double urand(void)
{
    rng_state ^= rng_state << 13;
    rng_state ^= rng_state >> 7;
    rng_state ^= rng_state << 17;
    return (double)(rng_state >> 11) * (1.0 / 9007199254740992.0);
}

static int check_edt(int X, int Y, int Z, double density, int nthreads)
{
    const int64_t N = (int64_t)X * Y * Z;
    uint8_t *occ = calloc((size_t)N, 1);
    int32_t *sq = malloc(sizeof(int32_t) * (size_t)N), *ix = malloc(sizeof(int32_t) * (size_t)N);
    int32_t *bsq = malloc(sizeof(int32_t) * (size_t)N), *bix = malloc(sizeof(int32_t) * (size_t)N);
    int bad = 0;
    for (int64_t i = 0; i < N; i++) occ[i] = urand() < density;
    int64_t *all = malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t i = 0; i < N; i++) all[i] = i;
    oracle_edt(occ, X, Y, Z, sq, ix, nthreads);
    oracle_edt_brute(occ, X, Y, Z, all, N, bsq, bix, nthreads);
    free(all);
    for (int64_t i = 0; i < N && !bad; i++) {
        if (sq[i] != bsq[i]) bad = 1;
        if (bsq[i] == INT32_MAX) {
            if (ix[i] != -1) bad = 1;
            continue;
        }
        if (ix[i] < 0 || ix[i] >= N || !occ[ix[i]]) {
            bad = 1;
            continue;
        }
        const int64_t dx = i % X - ix[i] % X, dy = (i / X) % Y - (ix[i] / X) % Y, dz = i / ((int64_t)X * Y) - ix[i] / ((int64_t)X * Y);
        if (dx * dx + dy * dy + dz * dz != sq[i]) bad = 1;
    }
    if (bad) fprintf(stderr, "EDT mismatch at %dx%dx%d density %g\n", X, Y, Z, density);
    free(occ); free(sq); free(ix); free(bsq); free(bix);
    return bad;
}

int main(void)
{
    int bad = 0;
    const int shapes[][3] = {{16, 16, 16}, {1, 1, 40}, {40, 1, 1}, {1, 30, 1}, {7, 5, 3}, {33, 17, 9}, {1, 1, 1}};
    const double dens[] = {0.0, 0.001, 0.05, 0.5, 1.0};
    for (size_t s = 0; s < sizeof(shapes) / sizeof(shapes[0]); s++)
        for (size_t d = 0; d < sizeof(dens) / sizeof(dens[0]); d++)
            bad |= check_edt(shapes[s][0], shapes[s][1], shapes[s][2], dens[d], 1 + (int)(d % 2) * 3);

    /* insertion of points (with a pose, NaN, outside, on the upper face) and links */
    const int X = 20, Y = 12, Z = 9;
    const float vs = 0.05f, origin[3] = {-0.1f, 0.2f, 0.0f};
    uint8_t *env = calloc(X * Y * Z, 1), *self = calloc(X * Y * Z, 1);
    const int64_t n = 4000;
    float *xyz = malloc(sizeof(float) * 3 * n);
    for (int64_t i = 0; i < 3 * n; i++) xyz[i] = (float)(urand() * 1.6 - 0.4);
    xyz[0] = NAN;
    xyz[4] = origin[1] + Y * vs;   /* upper face: outside */
    const float T[12] = {0, -1, 0, 0.3f, 1, 0, 0, 0.1f, 0, 0, 1, 0.05f};
    const int n_links = 2;
    const int64_t offs[3] = {0, 300, 700};
    float *pts = malloc(sizeof(float) * 3 * 700);
    for (int i = 0; i < 3 * 700; i++) pts[i] = (float)(urand() * 0.3);
    const float poses[24] = {1, 0, 0, 0.1f, 0, 1, 0, 0.3f, 0, 0, 1, 0.1f, 0, 0, 1, 0.2f, 0, 1, 0, 0.3f, -1, 0, 0, 0.35f};
    const int64_t nl = oracle_insert_links(self, X, Y, Z, vs, origin, n_links, pts, offs, poses, 0x3u);
    const int64_t np = oracle_insert_points(env, self, X, Y, Z, vs, origin, xyz, n, T, 1);
    const int64_t np2 = oracle_insert_points(env, self, X, Y, Z, vs, origin, xyz, n, NULL, 0);
    if (nl < 0 || np < 0 || np2 < 0 || np > n || np2 > n) bad = 1;

    /* query, including centres outside the grid and an empty map */
    int32_t *sq = malloc(sizeof(int32_t) * X * Y * Z), *ix = malloc(sizeof(int32_t) * X * Y * Z);
    oracle_edt(env, X, Y, Z, sq, ix, 2);
    float centres[3 * 8], radii[8];
    for (int i = 0; i < 24; i++) centres[i] = (float)(urand() * 1.8 - 0.5);
    centres[3] = NAN;
    for (int i = 0; i < 8; i++) radii[i] = 0.05f;
    sphere_out out[8];
    oracle_query(sq, ix, X, Y, Z, vs, origin, centres, radii, 8, out);
    memset(env, 0, X * Y * Z);
    oracle_edt(env, X, Y, Z, sq, ix, 1);
    oracle_query(sq, ix, X, Y, Z, vs, origin, centres, radii, 8, out);
    for (int i = 0; i < 8; i++)
        if (out[i].status == 0) bad = 1;   /* an empty map reports no nearest voxel */

    free(env); free(self); free(xyz); free(pts); free(sq); free(ix);
    if (!bad) printf("sanitized oracle run ok\n");
    return bad;
}
