/*
 * vedt.h -- C ABI of the B300-native exact voxel distance-map library.
 *
 * The calls follow the control cycle of "Real Time Collision Avoidance with
 * GPU-Computed Distance Maps" (arXiv 2407.02363), Alg. 2:
 *   line 1   initialise the self map M_S and environment map M_I  -> vedt_map_create
 *   line 4   ClearMap                                               -> vedt_clear
 *   line 5-6 UpdateLinks(q) + Insert(O_Lk) into M_S                 -> vedt_insert_links / vedt_insert_robot
 *   line 7   Insert(Point_Cloud) into M_I (robot points removed)    -> vedt_insert_pointcloud
 *   line 8   ForwardKinematics of the sphere centres                -> vedt_fk, vedt_sphere_centres (host)
 *   line 9   PBA_EDT(M_S, M_I): exact EDT, Sec. III-C, Alg. 1        -> vedt_compute_edt
 *   line 10  ExtractClosestObstaclePose, Eq. (dist), Alg. 3 l.3-4   -> vedt_query_spheres
 *
 * Conventions for every call:
 *  - Grids are X x Y x Z cubic voxels of edge voxel_size metres; voxel (x, y, z) has
 *    linear index x + X*(y + Y*z) (x fastest).  World point p lies in voxel
 *    floor((p - origin) / voxel_size) computed in fp32 (one rounded subtraction, one
 *    rounded division); it is inside iff 0 <= v < dims on every axis (points on the
 *    upper face and NaN points are outside).  1 <= X, Y, Z <= VEDT_MAX_DIM.
 *  - Occupancy grids are uint8 (nonzero = occupied).  The distance field is int32
 *    squared distance in voxel units plus int32 linear index of a nearest occupied
 *    voxel.  Where several occupied voxels are equally near, any of them may be
 *    returned.  An empty map yields sqdist = INT32_MAX and idx = -1 everywhere.
 *  - Calls are asynchronous and ordered on the map's CUDA stream unless stated
 *    otherwise.  Pointers named *_dev are device pointers, *_host host pointers.
 *    The caller owns every pointer it passes and keeps it valid until the stream work
 *    that uses it has completed.  The map owns its grids, fields and scratch.
 *  - Every call returns a vedt_status and never throws across the ABI.  Argument
 *    errors are detected on the host before any launch (VEDT_EINVAL).  A bounded wait
 *    that expires inside a kernel sets an error word that the next synchronising call
 *    reports (VEDT_ETIMEOUT).
 */
#ifndef VEDT_H
#define VEDT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VEDT_MAX_DIM 1024
#define VEDT_MAX_LINKS 16
#define VEDT_MAX_JOINTS 15

typedef enum {
    VEDT_OK = 0,
    VEDT_EINVAL = -1,    /* bad argument (null handle, dims, sizes, mask, ...)          */
    VEDT_ENOMEM = -2,    /* device or host allocation failed                           */
    VEDT_ECUDA = -3,     /* a CUDA runtime/driver call failed                          */
    VEDT_ETIMEOUT = -4,  /* a bounded in-kernel wait expired; results are invalid      */
    VEDT_EBUSY = -5,     /* not enough free device memory to admit the request         */
    VEDT_ENOTSUP = -6    /* request outside what this build supports                   */
} vedt_status;

/* which map(s) a call acts on */
enum { VEDT_MAP_ENV = 1, VEDT_MAP_SELF = 2, VEDT_MAP_BOTH = 3 };

/* sphere query status */
enum { VEDT_SPHERE_OK = 0, VEDT_SPHERE_OUTSIDE = 1, VEDT_SPHERE_EMPTY = 2 };

typedef struct vedt_map vedt_map;

/* Result of one sphere against one map (32 bytes). */
typedef struct {
    int32_t sqdist;      /* squared voxel distance at the centre's voxel (-1 if outside)  */
    int32_t idx;         /* linear index of the nearest occupied voxel O_i (-1 if none)   */
    float dist;          /* x_ci of Eq. (dist) in metres: voxel_size * sqrtf(sqdist)      */
    float clearance;     /* dist - sphere radius (Eq. (ref): >= 0 means no collision)     */
    float nearest[3];    /* world centre of voxel idx: origin + (v + 0.5) * voxel_size     */
    int32_t status;      /* VEDT_SPHERE_OK / _OUTSIDE (dist NaN) / _EMPTY (dist +inf)      */
} vedt_sphere_result;

/* Serial kinematic chain for vedt_fk / vedt_insert_robot.  Link 0 is the static body,
 * at `base` (3x4 row-major rotation | translation) in the world.  Joint k (1..n) sits
 * at offset[k-1] (3x4) in link k-1's frame and turns link k about that frame's z axis:
 * T_0 = base, T_k = T_(k-1) * offset_k * Rz(q_k). */
typedef struct {
    int32_t n_joints;                       /* 1 .. VEDT_MAX_JOINTS                    */
    double base[12];
    double offset[VEDT_MAX_JOINTS][12];
} vedt_chain;

/* ---- lifecycle (Alg. 2 line 1) ---------------------------------------------------- */

/* Creates M_I (environment) and M_S (self) grids of dims[3] = {X, Y, Z} voxels with
 * edge voxel_size > 0 and world min corner origin[3], plus both distance fields and
 * the EDT scratch; all device memory is allocated here (about 12*X*Y*Z bytes per grid
 * for dims <= 256, 15*X*Y*Z above).  `stream` is a cudaStream_t (NULL = legacy default
 * stream).  Grids start cleared.  *out receives the handle.  Errors: EINVAL, ENOMEM,
 * ECUDA. */
vedt_status vedt_map_create(const int32_t dims[3], float voxel_size, const float origin[3],
                            void *stream, vedt_map **out);

/* Frees all device memory of the map (synchronises its stream first).  NULL is a no-op. */
vedt_status vedt_map_destroy(vedt_map *map);

/* Rebinds the map to another stream (cudaStream_t); later calls are ordered there. */
vedt_status vedt_map_set_stream(vedt_map *map, void *stream);

/* Bands per line of EDT passes Y and Z: the m2 / m3 banding of Alg. 1 (Sec. III-C), and
 * the band ablation of Tab. 2 (PBA with m3 = 8 against PBA-naive, one band).  Each line
 * of a 32-column tile is cut into `bands` equal bands, each built by its own warp, then
 * joined.  Results do not depend on it; speed does.  0 restores the default (4 bands;
 * once a dim exceeds 256, 4 bands for lines up to 256 and 8 above).  Grids with every dim
 * <= 256 take 1, 2, 4 or 8, larger grids 4 or 8.  Applies to both grids from the next
 * vedt_compute_edt on.  Errors: EINVAL (NULL map, other values). */
vedt_status vedt_map_set_bands(vedt_map *map, int bands);

/* Tile shape of pass Z (Alg. 1 Step 4; a launch shape, the fields do not depend on it):
 * cols_x = 8 makes each warp's 32 columns an 8 x 4 patch of (x, y), cols_x = 32 a row of
 * 32 x-adjacent columns, 0 the default (8 x 4 if X is a multiple of 8, else 32 x 1).
 * Synchronises the map's streams and
 * rewrites its launch tables; a CUDA graph that holds this map's EDT launches must be
 * recorded again.  Errors: EINVAL (NULL map, other values), ECUDA. */
vedt_status vedt_map_set_tile_z(vedt_map *map, int cols_x);

/* The map's current pass-Z tile width (8 or 32; 0 for a NULL map). */
int vedt_map_tile_z(const vedt_map *map);

/* Bayesian occupancy of M_I (Sec. III-A names a Bayesian per-voxel update and gives
 * no model), in integer log-odds.  With on = 1 the map keeps an int8 log-odds value per
 * voxel of M_I, 0 (unknown) at the start.  Each
 * vedt_update_occupancy turns the current M_I (the voxels this frame's points landed in:
 * hits; all others: misses, no ray casting) into L <- clamp(L + l_hit | L - l_miss,
 * l_min, l_max) and sets M_I to L >= threshold.  vedt_frame / _host run it after the
 * point insertion (inside M_I's pass X when every dim is <= 256 and the map is not
 * incremental).  0 <= l_hit, l_miss <= 255; -128 <= l_min <= 0 <= l_max <= 127;
 * l_min < threshold (a threshold above l_max leaves M_I empty).
 * on = 0 frees the log-odds; enabling again restarts from 0.  Synchronises the map's
 * streams.  Errors: EINVAL, ENOMEM, ECUDA. */
vedt_status vedt_map_set_logodds(vedt_map *map, int on, int l_hit, int l_miss, int l_min, int l_max,
                                 int threshold);

/* The log-odds update of M_I from its current occupancy (see vedt_map_set_logodds),
 * asynchronous on the map's stream.  Errors: EINVAL (NULL map, log-odds off). */
vedt_status vedt_update_occupancy(vedt_map *map);

/* Incremental EDT (on = 1): vedt_compute_edt first compares each selected grid's
 * occupancy with a device snapshot taken at that grid's last EDT (one extra read of the
 * grid and of the snapshot, a write of the snapshot where they differ) and skips all
 * three passes of a grid whose occupancy is unchanged, leaving its fields as they are.
 * The fields are then still exact: the EDT is a function of the occupancy alone.  This
 * is the static-scene reuse of Sec. IV (a static scene needs one EDT while the arm
 * moves), decided on the device each call.  Enabling allocates the snapshots (2 x the
 * occupancy bytes) and the next EDT of each grid recomputes; on = 0 frees them.  A batch
 * EDT over the map also forces the next incremental EDT to recompute.  Synchronises the
 * map's stream.  Errors: EINVAL, ENOMEM, ECUDA. */
vedt_status vedt_map_set_incremental(vedt_map *map, int on);

/* After the map's stream drains: out[0] (and out[1] for VEDT_MAP_BOTH, env first) = 1
 * if the last vedt_compute_edt of that grid recomputed it, 0 if it was skipped as
 * unchanged (always 1 when the map is not incremental).  Synchronises.  Errors: EINVAL. */
vedt_status vedt_map_edt_recomputed(vedt_map *map, int which, int32_t *out);

/* Reports dims, voxel size and origin (any output may be NULL). */
vedt_status vedt_map_info(const vedt_map *map, int32_t dims_out[3], float *voxel_size_out,
                          float origin_out[3]);

/* ---- per-frame steps ---------------------------------------------------------------- */

/* ClearMap (Alg. 2 line 4; Tab. 1 "Clear Map"): zeroes the occupancy of the selected
 * map(s) (`which` = VEDT_MAP_ENV / _SELF / _BOTH). */
vedt_status vedt_clear(vedt_map *map, int which);

/* Insert(Point_Cloud) (Alg. 2 line 7; Sec. III-A).  xyz_dev: n_points x 3 fp32 device
 * array (sensor frame if T_world_sensor_host != NULL, else world).  T_world_sensor_host:
 * optional 3x4 fp32 row-major pose applied as w_a = ((T_a0 p_x + T_a1 p_y) + T_a2 p_z)
 * + T_a3 in fp32 without FMA.  Points outside the grid are dropped; with filter_self != 0
 * points whose voxel is occupied in M_S are dropped (robot-point removal, Sec. III-A).
 * counts_dev (nullable, device int64[3]) is incremented by {written, outside, filtered}.
 * n_points = 0 is valid.  Errors: EINVAL (null map/xyz with n > 0, n < 0). */
vedt_status vedt_insert_pointcloud(vedt_map *map, const float *xyz_dev, int64_t n_points,
                                   const float *T_world_sensor_host, int filter_self,
                                   int64_t *counts_dev);

/* As vedt_insert_pointcloud, but point i is inserted only if keep_dev[i] != 0 (device
 * uint8 per point, e.g. the output of vedt_sor_filter; NULL keeps every point).  Dropped
 * points are not counted.  Errors: EINVAL. */
vedt_status vedt_insert_pointcloud_masked(vedt_map *map, const float *xyz_dev, int64_t n_points,
                                          const float *T_world_sensor_host, int filter_self,
                                          const uint8_t *keep_dev, int64_t *counts_dev);

/* Registers the offline link voxel models (Sec. III-A): link k's model is
 * link_xyz_host[k], n_vox[k] fp32 xyz points in the link frame.  Copied to the device
 * once (synchronously); replaces any earlier registration.  Link 0 is the static body.
 * 1 <= n_links <= VEDT_MAX_LINKS, n_vox[k] >= 0.  Errors: EINVAL, ENOMEM, ECUDA. */
vedt_status vedt_register_links(vedt_map *map, int n_links, const float *const *link_xyz_host,
                                const int64_t *n_vox);

/* UpdateLinks + Insert(O_Lk) (Alg. 2 lines 5-6; Sec. III-E): moves every registered
 * link k with bit k set in link_mask by poses_host[12k .. 12k+12) (3x4 fp32 row-major
 * R | t, same arithmetic as above) and marks the voxels in M_S.  The set of links in
 * the mask is the self-collision obstacle O_L of Eq. (selfclink).  Errors: EINVAL (no
 * links registered, mask names an unregistered link). */
vedt_status vedt_insert_links(vedt_map *map, const float *poses_host, uint32_t link_mask);

/* Forward kinematics on the host in fp64 (Alg. 2 lines 5 and 8): poses_out receives
 * (chain->n_joints + 1) 3x4 row-major transforms T_0 .. T_n (see vedt_chain).  Each
 * matrix entry is summed left to right without FMA.  Errors: EINVAL. */
vedt_status vedt_fk(const vedt_chain *chain, const double *q, double *poses_out);

/* vedt_fk for n joint vectors q[n][n_joints]: poses_out[n][n_joints + 1][12]. */
vedt_status vedt_fk_batch(const vedt_chain *chain, const double *q, int64_t n, double *poses_out);

/* C_i <- FK(q) (Alg. 2 line 8): world centres of m bounding spheres.  Sphere i sits on
 * link link_of[i] (0 .. chain->n_joints; 0 = the static body) at local[3i .. 3i+3) in
 * that link's frame (metres).  With T = vedt_fk(chain, q)[link_of[i]] (fp64) each
 * coordinate is c_a = ((T_a0 l_0 + T_a1 l_1) + T_a2 l_2) + T_a3, summed left to right
 * without FMA, then rounded to fp32 into centres_out[3i + a] (host memory, caller-owned,
 * m x 3 floats).  m = 0 writes nothing.  Errors: EINVAL (null pointer with m > 0, m < 0,
 * a link index outside 0 .. n_joints, an invalid chain). */
vedt_status vedt_sphere_centres(const vedt_chain *chain, const double *q, int m, const int32_t *link_of,
                                const double *local, float *centres_out);

/* vedt_sphere_centres for n joint vectors q[n][n_joints]: centres_out[n][m][3]. */
vedt_status vedt_sphere_centres_batch(const vedt_chain *chain, const double *q, int64_t n, int m,
                                      const int32_t *link_of, const double *local, float *centres_out);

/* vedt_fk followed by rounding the poses to fp32 and vedt_insert_links(link_mask).
 * The chain must have n_joints + 1 <= registered links.  Errors: as both calls. */
vedt_status vedt_insert_robot(vedt_map *map, const vedt_chain *chain, const double *q,
                              uint32_t link_mask);

/* PBA_EDT (Alg. 2 line 9; Sec. III-C, Alg. 1): exact squared Euclidean distance
 * transform of the selected occupancy grid(s) with a nearest occupied voxel per voxel,
 * as three separable sweeps (rows along x; lower envelopes along y, then along z). */
vedt_status vedt_compute_edt(vedt_map *map, int which);

/* ExtractClosestObstaclePose + x_ci = |O_i - C_i| (Alg. 2 line 10; Eq. (dist); Alg. 3
 * lines 3-4) at the voxels holding the m sphere centres.  centres_host: m x 3 fp32
 * world; radii_host: m fp32.  out_host: m results per selected map, ENV block first
 * when which = VEDT_MAP_BOTH (2m results).  Synchronises the stream and reports any
 * pending in-kernel error.  1 <= m <= 4096.  Errors: EINVAL, ETIMEOUT, ECUDA. */
vedt_status vedt_query_spheres(vedt_map *map, const float *centres_host, const float *radii_host,
                               int m, int which, vedt_sphere_result *out_host);

/* Same query on device buffers, asynchronous (no synchronisation, no error check). */
vedt_status vedt_query_spheres_dev(vedt_map *map, const float *centres_dev, const float *radii_dev,
                                   int m, int which, vedt_sphere_result *out_dev);

/* ---- one control cycle ------------------------------------------------------------------- */

/* Alg. 2 lines 4-10 in one call on device buffers, asynchronous: vedt_clear(BOTH),
 * vedt_insert_robot(chain, q, link_mask) (skipped if chain == NULL), vedt_insert_pointcloud
 * (xyz_dev, n_points, T_world_sensor_host, filter_self = 1), the EDT of both maps and
 * vedt_query_spheres_dev(centres_dev, radii_dev, m, BOTH, out_dev) (skipped if m == 0).
 * M_S is final once the links are in, so its EDT runs on a side stream owned by the map,
 * concurrently with the point insertion and M_I's EDT on the map's stream; the query
 * waits for both, and the call's work is complete when the map's stream is (one frame
 * never overlaps the next).  While per-kernel timing is on, the same launches run one
 * after another on the map's stream.  Errors: as the individual calls. */
vedt_status vedt_frame(vedt_map *map, const float *xyz_dev, int64_t n_points,
                       const float *T_world_sensor_host, const vedt_chain *chain, const double *q,
                       uint32_t link_mask, const float *centres_dev, const float *radii_dev, int m,
                       vedt_sphere_result *out_dev);

/* The same cycle from host buffers: copies xyz_host (n_points x 3 fp32; page-locked memory
 * makes the copy asynchronous) into one of the map's two device staging buffers (grown on
 * demand, ENOMEM if that fails) on the map's own copy stream, and centres/radii into one
 * of four page-locked slots of the map that the query kernel reads in place (the call
 * waits for the frame four back if that one still reads the slot); runs vedt_frame on the
 * map's stream once the upload has landed, delivers
 * the 2m results (ENV block first) to out_host and synchronises the stream, reporting any
 * pending in-kernel error.  If out_host is page-locked memory the device can address (for
 * instance from cudaHostAlloc), the query kernel writes the results into it directly;
 * otherwise they are copied after the frame.  1 <= m <= 4096 or m == 0. */
vedt_status vedt_frame_host(vedt_map *map, const float *xyz_host, int64_t n_points,
                            const float *T_world_sensor_host, const vedt_chain *chain, const double *q,
                            uint32_t link_mask, const float *centres_host, const float *radii_host,
                            int m, vedt_sphere_result *out_host);

/* ---- batches of maps ---------------------------------------------------------------------- */

/* A batch runs the per-frame pipeline of Alg. 2 (lines 4-10) for many independent maps of
 * uneven extents at once: each step is one launch over all maps, and the EDT of every
 * grid in the batch is one persistent launch whose work items (rows for the row sweep,
 * 32-column tiles for the two envelope sweeps) are handed out in order, each envelope
 * tile waiting (bounded) only for its own grid's previous sweep.  Maps with a dimension
 * > 256 form a second persistent launch.  The batch references (does not own) its maps;
 * they must outlive it.  All batch calls are ordered on the batch's stream. */
typedef struct vedt_batch vedt_batch;

vedt_status vedt_batch_create(vedt_map *const *maps, int n_maps, void *stream, vedt_batch **out);
vedt_status vedt_batch_destroy(vedt_batch *batch);

/* Launch-shape knobs explored by the autotuner: ctas_per_sm (0 = occupancy maximum) and
 * rows_per_item (pass-X rows per work item) of the persistent EDT, or persistent = 0 for
 * three plain launches (one per sweep) over all grids.  Results never depend on them.
 * Drops a recorded graph. */
vedt_status vedt_batch_set_tuning(vedt_batch *batch, int ctas_per_sm, int rows_per_item, int persistent);

/* Bands per line of passes Y and Z for the batch's EDT, as vedt_map_set_bands (Alg. 1's
 * m2 / m3): 0 = the default, 1, 2, 4 or 8 for the grids with every dim <= 256 (the maps
 * with a larger dim keep 4 / 8 by line length, or take 4 or 8).  Applies to the plain
 * and the persistent launches.  Drops a recorded graph.  Errors: EINVAL. */
vedt_status vedt_batch_set_bands(vedt_batch *batch, int bands);

/* Pass-Z tile shape of the batch's grids with every dim <= 256, as vedt_map_set_tile_z
 * (the default looks at every such grid's X; the batch's larger grids keep 32 x 1, the
 * shape of their persistent kernel).  Applies to the plain and the persistent launches.  Synchronises the batch's stream, rewrites its launch tables and drops a
 * recorded graph.  Errors: EINVAL, ECUDA. */
vedt_status vedt_batch_set_tile_z(vedt_batch *batch, int cols_x);

/* The batch's current pass-Z tile width for its grids with every dim <= 256 (8 or 32; 0
 * if it has none). */
int vedt_batch_tile_z(const vedt_batch *batch);

/* PBA_EDT (Alg. 2 line 9) of the selected grids (default both) of every map in the batch. */
vedt_status vedt_batch_compute_edt(vedt_batch *batch);

/* Restricts the batch EDT to one grid of every map (VEDT_MAP_ENV / _SELF) or both
 * (default); the skipped grid's field keeps its old contents.  Drops a recorded graph. */
vedt_status vedt_batch_set_grids(vedt_batch *batch, int which);

/* Offline link models shared by every map of the batch (same robot, own joint states);
 * as vedt_register_links. */
vedt_status vedt_batch_register_links(vedt_batch *batch, int n_links, const float *const *link_xyz_host,
                                      const int64_t *n_vox);

/* Inputs of the next frame.  xyz_dev: world-frame fp32 points of all maps, map i owning
 * points [offsets_host[i], offsets_host[i+1]) (offsets_host[0] = 0, n_maps + 1 entries).
 * poses_host: n_maps x n_links x 12 fp32 link poses.  centres_dev: n_maps x m x 3 fp32
 * sphere centres, radii_dev: m fp32 radii, out_dev: n_maps x 2 x m results (per map the
 * environment block, then the self block).  Device pointers are kept, not copied; poses
 * and offsets are copied to the device before the call returns.  Once a graph is recorded
 * the device pointers, m, link_mask must stay the same and no map may exceed the point
 * count it had at recording (EINVAL otherwise). */
vedt_status vedt_batch_set_frame(vedt_batch *batch, const float *xyz_dev, const int64_t *offsets_host,
                                 const float *poses_host, uint32_t link_mask, const float *centres_dev,
                                 const float *radii_dev, int m, vedt_sphere_result *out_dev);

/* One frame for every map: clear both grids, insert links (link_mask) into M_S, insert
 * the points into M_I with robot-point removal, EDT of all grids, sphere query. */
vedt_status vedt_batch_run(vedt_batch *batch);

/* Records vedt_batch_run as a CUDA graph (needs a non-default stream); vedt_batch_replay
 * launches it, reading the frame inputs current at replay time. */
vedt_status vedt_batch_capture(vedt_batch *batch);
vedt_status vedt_batch_replay(vedt_batch *batch);

/* Synchronises the batch's stream; ETIMEOUT if an in-kernel wait expired. */
vedt_status vedt_batch_check(vedt_batch *batch);

/* Asynchronous vedt_frame_host: the frame and the delivery of the 2m results (written by
 * the query kernel into a page-locked out_host, else copied after the frame) are queued on
 * the map's stream and the call returns at once.  The cloud upload goes to the staging
 * buffer the previous frame did not use, on the map's copy stream, after the frame that
 * last read that buffer has finished; so a frame queued behind a running one uploads while
 * the earlier one computes.  xyz_host and out_host must stay valid until vedt_frame_done
 * reports completion (page-locked memory keeps the copies asynchronous); centres/radii are
 * copied (into the map's page-locked slot of this frame) before the call returns, which
 * waits only if the frame queued four calls earlier is still running. */
vedt_status vedt_frame_host_async(vedt_map *map, const float *xyz_host, int64_t n_points,
                                  const float *T_world_sensor_host, const vedt_chain *chain, const double *q,
                                  uint32_t link_mask, const float *centres_host, const float *radii_host,
                                  int m, vedt_sphere_result *out_host);

/* VEDT_OK once every frame queued by vedt_frame_host_async on this map has completed,
 * VEDT_EBUSY while one is still running, ETIMEOUT/ECUDA on failure.  Never blocks. */
vedt_status vedt_frame_done(vedt_map *map);

/* Device memory a map of these dims allocates (bytes), for admission control. */
int64_t vedt_map_bytes(const int32_t dims[3]);

/* Free and total device memory of the current device (cudaMemGetInfo). */
vedt_status vedt_device_memory(int64_t *free_bytes, int64_t *total_bytes);

/* ---- access ---------------------------------------------------------------------------- */

/* Borrowed device pointers to the selected map's fields (which = ENV or SELF), valid
 * until the map is destroyed; contents change with later calls. */
vedt_status vedt_get_field(vedt_map *map, int which, const int32_t **sqdist_dev,
                           const int32_t **idx_dev);
vedt_status vedt_get_occupancy(vedt_map *map, int which, uint8_t **occ_dev);

/* Synchronises the map's stream and returns ETIMEOUT/ECUDA if any kernel flagged an
 * error since the last check (and clears the flag), else OK. */
vedt_status vedt_check(vedt_map *map);

/* Per-kernel timing with CUDA events on the map's stream.  enable != 0 starts
 * recording an event pair around every launch; vedt_kernel_times synchronises and adds
 * the accumulated milliseconds and launch counts of each kernel kind into ms_out /
 * count_out (arrays of VEDT_NUM_KERNELS, nullable), then resets the accumulators. */
enum { VEDT_K_CLEAR = 0, VEDT_K_INSERT_LINKS, VEDT_K_INSERT_POINTS, VEDT_K_EDT_X,
       VEDT_K_EDT_Y, VEDT_K_EDT_Z, VEDT_K_QUERY, VEDT_K_OCCUPANCY, VEDT_NUM_KERNELS };
vedt_status vedt_set_timing(vedt_map *map, int enable);
vedt_status vedt_kernel_times(vedt_map *map, double *ms_out, int64_t *count_out);

/* ---- learned self-distance surrogate (not in the paper) ----------------------------------- */

/* A BF16 MLP  [sin q, cos q] (14) -> 4 x (Linear 256 + ReLU) -> Linear 24  predicting the
 * 24 per-sphere self-collision distances x_si of Eq. (selftaskvar) (metres) from the 7
 * joint angles, trained on labels from the exact self-map EDT.  Every matrix product runs
 * on the tensor cores (tcgen05.mma, bf16 operands, fp32 accumulation in tensor memory).
 * Parameters are exchanged as one flat fp32 array, layer by layer W_l (out x in,
 * row-major) then b_l (out): vedt_mlp_num_params() values. */
typedef struct vedt_mlp vedt_mlp;

int64_t vedt_mlp_num_params(void);
/* batch_capacity: largest batch any later call may pass (rounded up to 128). */
vedt_status vedt_mlp_create(int batch_capacity, void *stream, vedt_mlp **out);
vedt_status vedt_mlp_destroy(vedt_mlp *net);
/* Loads fp32 parameters (host), resets the AdamW moments and step count; synchronises. */
vedt_status vedt_mlp_set_params(vedt_mlp *net, const float *params_host, int64_t count);
vedt_status vedt_mlp_get_params(vedt_mlp *net, float *params_host, int64_t count);
/* Training state for checkpoint / resume: the parameters, the AdamW first and second
 * moments (each `count` = vedt_mlp_num_params() fp32 values in the flat layout, host
 * buffers) and the step count.  get synchronises; set loads all of it (the next
 * vedt_mlp_train_step continues from there) and synchronises.  Errors: EINVAL (NULL
 * pointers, wrong count, negative step), ECUDA. */
vedt_status vedt_mlp_get_state(vedt_mlp *net, float *params_host, float *m1_host, float *m2_host, int64_t count,
                               int64_t *step);
vedt_status vedt_mlp_set_state(vedt_mlp *net, const float *params_host, const float *m1_host,
                               const float *m2_host, int64_t count, int64_t step);
/* q_dev: B x 7 fp32 joint angles; out_dev: B x 24 fp32 predicted distances.  Async.
 * One persistent fused kernel, one CTA per SM: each CTA keeps two 128-row activation
 * tiles in shared memory through all five layers, with one fp32 accumulator per tile in
 * tensor memory, and streams pre-packed weight chunks through a ring of shared-memory
 * stages. */
vedt_status vedt_mlp_forward(vedt_mlp *net, const float *q_dev, int B, float *out_dev);
/* The same forward as one GEMM launch per layer (the training path's kernels). */
vedt_status vedt_mlp_forward_layers(vedt_mlp *net, const float *q_dev, int B, float *out_dev);
/* Masked mean-squared-error loss on (q_dev, y_dev B x 24, mask_dev B x 24 or NULL):
 * gradient of every parameter (host, flat layout) and the loss; synchronises. */
vedt_status vedt_mlp_grads(vedt_mlp *net, const float *q_dev, const float *y_dev, const float *mask_dev, int B,
                           float *grads_host, int64_t count, float *loss_host);
/* One AdamW step (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay wd) on that loss;
 * loss_sums_dev (nullable, 2 floats) receives {sum of squared errors, mask count}.  Async. */
vedt_status vedt_mlp_train_step(vedt_mlp *net, const float *q_dev, const float *y_dev, const float *mask_dev, int B,
                                float lr, float wd, float *loss_sums_dev);
/* Synchronises; ETIMEOUT if an in-kernel wait expired. */
vedt_status vedt_mlp_check(vedt_mlp *net);

/* ---- statistical outlier filter of the raw cloud (Sec. III-A) ---------------------------- */

/* Sec. III-A filters the raw cloud by each point's distances to its neighbours before it
 * is transformed and inserted; the paper gives no parameters.  Here: d_i = mean Euclidean
 * distance of point i to its k nearest other valid points (valid: all coordinates
 * finite), and point i is kept iff it is valid and d_i <= mean(d) + std_mul * std(d) over
 * the valid points (sample standard deviation).  Exact kNN; squared distances in float64
 * from the float32 coordinates, the k square roots summed in ascending order, the cloud's
 * sums kept exactly as 128-bit fixed-point integers (units of 2^-80 m), so the decision is
 * reproducible bit for bit.  Distances must stay below 2^20 (metres) for exact sums. */
typedef struct vedt_sor vedt_sor;

/* A filter for clouds of up to max_points points (device scratch of about 40 bytes per
 * point plus a cell grid of up to 2*max_points cells), ordered on `stream` (cudaStream_t).
 * Errors: EINVAL, ENOMEM, ECUDA. */
vedt_status vedt_sor_create(int64_t max_points, void *stream, vedt_sor **out);
vedt_status vedt_sor_destroy(vedt_sor *f);   /* synchronises; NULL is a no-op */

/* keep_dev[i] = 1 if point i (xyz_dev: n float32 triples on the device) is kept, else 0.
 * 1 <= k <= 64, std_mul finite, 0 <= n <= max_points.  Asynchronous on the filter's
 * stream; xyz_dev and keep_dev must stay valid until it completes.  Errors: EINVAL, ECUDA. */
vedt_status vedt_sor_filter(vedt_sor *f, const float *xyz_dev, int64_t n, int k, double std_mul,
                            uint8_t *keep_dev);

/* After the stream drains: stats_out = {mean, std, threshold} of the last filter call,
 * counts_out = {valid points, kept points} (either may be NULL).  Synchronises. */
vedt_status vedt_sor_stats(vedt_sor *f, double stats_out[3], int64_t counts_out[2]);

/* Borrowed device pointer to the last call's d_i (float64 per input point; entries of
 * invalid points are not written).  Valid until the next filter call or destroy. */
vedt_status vedt_sor_mean_distances(vedt_sor *f, const double **d_dev);

/* ---- EDT without device allocation -------------------------------------------------------- */

/* The paper has no counterpart to this call; it exists for callers that must not allocate
 * device memory once running: a hard real-time control loop (cudaMalloc may synchronise
 * the device and has no latency bound) or a process whose device memory is already
 * reserved by another allocator.  It computes the same exact EDT as vedt_compute_edt for
 * one grid: occ_dev (X*Y*Z uint8, layout as above) in, sqdist_dev and idx_dev (X*Y*Z
 * int32 each) out, all caller-owned device memory, on `stream` (cudaStream_t, NULL =
 * legacy default stream).  The call returns when its work on `stream` has finished (it
 * synchronises the stream and reads back the device error word), so it also refuses a
 * stream that is being captured (VEDT_ENOTSUP).  Scratch comes from one fixed array of
 * about 6.4 MB that the library keeps in every GPU's memory until the process exits: each
 * dimension must be <= 256 and ceil(X/32)*32*Y*Z <= 2^21 (a 128^3 grid fits), otherwise
 * the call returns VEDT_ENOTSUP without doing anything.  Each call looks the array up on
 * the current device (cudaGetSymbolAddress), so it is found again after a device reset.
 * Calls share the array and leave their scratch in it;
 * calls that may overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.
 * Errors: EINVAL (null pointer, dims < 1), ENOTSUP (grid larger than the scratch, stream
 * under capture), ECUDA (a CUDA error, or an index the bounds-checked build flagged),
 * ETIMEOUT (an in-kernel wait expired). */
vedt_status vedt_edt_noalloc(const uint8_t *occ_dev, int32_t X, int32_t Y, int32_t Z,
                             int32_t *sqdist_dev, int32_t *idx_dev, void *stream);

/* Failure-detection self-test: launches the bounded in-kernel wait used by the persistent
 * EDT on a counter that nothing increments, with `limit` polls (each followed by a ~64 ns
 * sleep).  Returns VEDT_ETIMEOUT when the wait expired and flagged the error word as it
 * should (the kernel then exits normally and the context stays usable), VEDT_OK if it did
 * not.  Synchronises `stream`. */
vedt_status vedt_selftest_wait(void *stream, uint32_t limit);

/* Human-readable text for a status code (static storage). */
const char *vedt_status_string(vedt_status s);

/* Library version string; the bounds-checked debug build (libvedt_debug.so, built with
 * -DVEDT_DEBUG_BOUNDS: the EDT passes check each index they compute and report a bad one
 * as VEDT_ECUDA from vedt_check) says "index checks". */
const char *vedt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VEDT_H */
