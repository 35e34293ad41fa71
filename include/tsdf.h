/*
 * tsdf.h — C ABI of the GB300 projective TSDF integration library.
 *
 * The library builds the TSDF layer of a sparse voxel map from depth images
 * (nvblox, Sec. IV "System architecture"): the map is a hash table from
 * integer 3D block coordinates to 8x8x8-voxel blocks stored contiguously in
 * GPU memory (Sec. IV-A "The Map"), and every frame is integrated by
 * allocating the blocks in view and running a per-voxel projective update
 * (Sec. IV-B "Frame Integration", Eq. 1-3).  Sensors follow the problem
 * statement (Sec. III): a depth image D: Omega -> d with Omega the pinhole
 * image plane (z-depth) or the LiDAR beam angles (range), taken at a pose
 * T_LC in SE(3) of the sensor in the layer frame.  On the same block
 * structure the library also keeps an occupancy or colour layer instead of
 * the TSDF (TSDF_LAYER_*), and derives from a TSDF layer its incremental
 * ESDF (Sec. IV-C, map_esdf_*) and a marching-cubes mesh (map_mesh).
 *
 * Conventions shared by every call:
 *  - All buffers are owned by the caller.  Pointers named *_dev are device
 *    pointers that must stay valid until the call's work on `cuda_stream`
 *    has finished; pointers named *_host are host memory.  Poses are host
 *    memory, row-major 4x4 doubles, read during the call (copied by value).
 *  - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).
 *    Calls return as soon as their work is enqueued, except those whose
 *    description says they synchronise or wait.
 *  - Argument errors are returned synchronously and enqueue nothing.
 *    Errors found on the device (pool or hash full, work list full) are
 *    sticky on the map and returned by map_sync() and by every later call;
 *    after TSDF_ERR_CAPACITY the map's contents are unspecified.  No call
 *    aborts, traps or waits without bound.
 *  - One map must not be used from two host threads at once.
 *  - Voxel indexing: voxel index g = floor(p / voxel_size) per axis; block
 *    b = floor(g / 8); local index l = g - 8 b, flattened x + 8 y + 64 z.
 *    Block coordinates must lie in [-2^20, 2^20).
 *  - Voxel values: D is the truncated signed distance in metres, W the
 *    accumulated weight; W = 0 means never updated.
 *
 * Precision: discrete decisions (blocks met by a band segment, pixel choice,
 * sample validity, the d_p >= -tau test, LiDAR cell choice) are taken in a
 * prescribed FP32 operation sequence; values are accumulated in FP32 and
 * stored in FP32, FP16 or 16-bit fixed point (TSDF_STORAGE_*).  Poses are composed in
 * FP64 on the host and passed to the GPU as FP32, relative to the block that
 * contains the sensor origin.
 */
#ifndef GB300_TSDF_H_
#define GB300_TSDF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsdf_map tsdf_map; /* opaque; created and owned by the library */

typedef enum {
  TSDF_OK = 0,
  TSDF_ERR_ARG = -1,      /* bad argument: nothing was enqueued              */
  TSDF_ERR_CUDA = -2,     /* a CUDA runtime call or launch failed             */
  TSDF_ERR_CAPACITY = -3, /* block pool, hash table or work list full         */
  TSDF_ERR_TIMEOUT = -4,  /* a bounded device wait gave up                    */
  TSDF_ERR_STATE = -5     /* call not valid in the map's current state        */
} tsdf_status;

/* Pinhole intrinsics (Eq. 2): u = fu x / z + cu, v = fv y / z + cv; pixel
 * (i, j) has its centre at (u, v) = (i, j). */
typedef struct {
  float fu, fv, cu, cv;
  int32_t width, height;
} tsdf_pinhole;

/* Spinning LiDAR (Eq. 3): n_az columns cover the full azimuth circle from
 * theta_start (radians, about +z); n_el rows cover polar angles
 * [phi_start, phi_start + el_fov] measured from +z, row 0 first.  Ranges
 * outside [min_range, max_range] or non-finite are invalid. */
typedef struct {
  int32_t n_az, n_el;
  float theta_start, phi_start, el_fov;
  float min_range, max_range;
} tsdf_lidar;

/* TSDF voxel storage (arithmetic is FP32 in every case).  FP32: D and W as
 * floats, 8 B per voxel.  FP16: D / tau and W as halves, 4 B per voxel.
 * FIXED16: D / tau as a 16-bit signed fixed-point fraction (32767 steps per
 * tau, rounded to nearest) and W as a half, 4 B per voxel.  Both 4-byte forms
 * hold integer weights up to 2048 exactly.  Each update rounds the stored D
 * once, so with the running average at the weight cap (a step of
 * (s - D) / (max_weight + 1)) the stored D can stay up to
 * (max_weight + 1) / 2 units of its last place from the exact average: FP16
 * units are 2^-11 tau for |D| >= tau / 2, fixed-point units a uniform
 * tau / 32767, so FIXED16 bounds that error by (max_weight + 1) / 65534 tau
 * (1.5e-3 tau at max_weight 100). */
enum { TSDF_STORAGE_FP32 = 0, TSDF_STORAGE_FP16 = 1, TSDF_STORAGE_FIXED16 = 2 };
/* Layers (Sec. IV-A: a map of co-located layers; Sec. IV-B: one update
 * functor per layer).  An occupancy layer holds one FP32 log-odds per voxel:
 * every voxel that passes the same projection test as the TSDF (d_p >= -tau)
 * adds l_free if it lies in front of the surface (d_p > 0) and l_occ
 * otherwise; `storage` is ignored, exported distances are the log-odds and
 * exported / queried weights are 0. */
/* A colour layer (Sec. III: colour images C: Omega -> R^3; Table I: colour
 * fusion) holds r, g, b and a colour weight per voxel (four FP32, 16 B):
 * integrate_color fuses a colour image registered to a depth image (same
 * intrinsics and pose); the depth image allocates the band like the TSDF,
 * and every voxel within tau of the surface on both sides
 * (-tau <= d_p <= tau) folds the colour of the pixel it projects to into a
 * running average with weight 1, weights summed up to max_weight.  Colour
 * maps take pinhole frames only; `storage` is ignored. */
enum { TSDF_LAYER_TSDF = 0, TSDF_LAYER_OCCUPANCY = 1, TSDF_LAYER_COLOR = 2 };
/* TSDF weighting functions (Sec. IV-B: w = f_w(d_p), constant or from the
 * sensor's error model), combinable: the weight is 1, times 1 / d_v^2 with
 * TSDF_WEIGHT_INV_SQUARE, times a linear drop-off from 1 at d_p = -dropoff to
 * 0 at d_p = -tau with TSDF_WEIGHT_DROPOFF.  Non-constant weights are not
 * integers: with FP16 storage W is then rounded to 11 significant bits. */
enum { TSDF_WEIGHT_CONSTANT = 0, TSDF_WEIGHT_INV_SQUARE = 1, TSDF_WEIGHT_DROPOFF = 2 };
enum { TSDF_SENSOR_PINHOLE = 0, TSDF_SENSOR_LIDAR = 1 };

/* Map options.  max_blocks: pool size in blocks (4 KiB per block in FP32,
 * 2 KiB in FP16 or FIXED16); hash_capacity: hash slots, rounded up to a power of two,
 * at least 2 * max_blocks (0 = that minimum).  lidar_nearest != 0 samples
 * LiDAR images at the nearest beam instead of guarded bilinear;
 * lidar_guard is the bilinear foreground/background threshold in metres
 * (<= 0: the truncation distance).  Launch-shape knobs (results do not
 * depend on them): alloc_tile_h is the pixel-tile height of the allocation
 * kernel, 16 or 32 (0 = chosen from the pixels per launch);
 * integrate_ctas_per_sm is the integration kernel's resident CTAs per SM
 * (0 = as many as fit).  For integrate_batch the first map's knobs apply.
 * layer selects the update functor (all maps of one integrate_batch call
 * must share layer and storage).  launch_mode: TSDF_LAUNCH_SPLIT (default)
 * runs each sub-batch of integrate_batch as an allocation launch and an
 * integration launch, overlapping one sub-batch's allocation with the
 * previous one's integration; TSDF_LAUNCH_FUSED runs each sub-batch as one
 * persistent, cooperative launch that allocates, waits at a bounded
 * grid-wide barrier (TSDF_ERR_TIMEOUT if it does not complete within about
 * a second) and integrates, sub-batches one after the other; it covers
 * single-map calls of TSDF layers with constant weighting and walk
 * statistics off, and other calls fall back to the split form.  Results do
 * not depend on the mode. */
enum { TSDF_LAUNCH_SPLIT = 0, TSDF_LAUNCH_FUSED = 1 };
typedef struct {
  int32_t storage;
  int64_t max_blocks;
  int64_t hash_capacity;
  int32_t lidar_nearest;
  float lidar_guard;
  int32_t alloc_tile_h;
  int32_t integrate_ctas_per_sm;
  int32_t layer;       /* TSDF_LAYER_TSDF, _OCCUPANCY or _COLOR */
  float l_occ, l_free; /* occupancy: log-odds added per update (0, 0: 0.85, -0.4) */
  int32_t weighting;   /* TSDF weight f_w, TSDF_WEIGHT_* flags (0 = constant 1) */
  float dropoff;       /* drop-off start behind the surface, m (<= 0: one voxel) */
  int32_t launch_mode; /* TSDF_LAUNCH_SPLIT or TSDF_LAUNCH_FUSED */
} tsdf_map_opts;

/* One frame of a batch.  `map` indexes the maps array of integrate_batch;
 * `kind` selects which intrinsics member is read; depth_dev is the image
 * (row-major [height][width] z-depth or [n_el][n_az] range, float32);
 * T_world_sensor is the sensor-to-layer pose T_LC; color_dev is the
 * registered colour image (uint32 [height][width], r in the low byte, then
 * g, b; the top byte is ignored): required for colour maps, NULL otherwise. */
typedef struct {
  int32_t map;
  int32_t kind;
  tsdf_pinhole pinhole;
  tsdf_lidar lidar;
  const float* depth_dev;
  double T_world_sensor[16];
  const uint32_t* color_dev;
} tsdf_frame_desc;

/*
 * map_create — an empty TSDF layer (Sec. IV-A) with voxel edge voxel_size
 * (metres, > 0), truncation distance tau = truncation_voxels * voxel_size
 * (the epsilon of Sec. IV-B) and weights summed up to max_weight (> 0).
 * Defaults: FP32 storage, 2^18 blocks.  Allocates device memory on the
 * current CUDA device.  Returns TSDF_ERR_ARG for bad sizes, TSDF_ERR_CUDA if
 * allocation fails; *out is set only on success.
 */
tsdf_status map_create(float voxel_size, int32_t truncation_voxels, float max_weight,
                       tsdf_map** out);

/* map_create_ex — as map_create with explicit options (NULL = defaults). */
tsdf_status map_create_ex(float voxel_size, int32_t truncation_voxels, float max_weight,
                          const tsdf_map_opts* opts, tsdf_map** out);

/*
 * integrate_depth — integrate one pinhole z-depth image (Sec. IV-B):
 * allocate every block met by the band segment z in [d - tau, d + tau] of a
 * valid pixel's ray (block-grid traversal after Amanatides & Woo), then for
 * every voxel of those blocks project its centre (Eq. 1, Eq. 2), sample the
 * nearest pixel, form d_p = d - z_v, skip the voxel if d_p < -tau, and fold
 * min(d_p, tau) into the weighted running average with weight 1, summing
 * weights up to max_weight.  depth_dev: float32 [height][width], z-depth in
 * metres, <= 0 or non-finite = invalid.  T_world_cam: camera-to-layer pose
 * (camera axes x right, y down, z forward).  Async on cuda_stream.
 */
tsdf_status integrate_depth(tsdf_map* map, const float* depth_dev, const tsdf_pinhole* intr,
                            const double T_world_cam[16], void* cuda_stream);

/*
 * integrate_lidar — integrate one spinning-LiDAR range image (Sec. IV-B,
 * Eq. 3): as integrate_depth with the band in range, d_v = |p_C| and the
 * sample taken by bilinear interpolation between the four surrounding beam
 * centres (azimuth wraps), skipped if any of the four is invalid or their
 * spread exceeds the guard threshold.  range_dev: float32 [n_el][n_az].
 */
tsdf_status integrate_lidar(tsdf_map* map, const float* range_dev, const tsdf_lidar* intr,
                            const double T_world_lidar[16], void* cuda_stream);

/*
 * integrate_color — integrate one registered depth + colour pair into a
 * colour map (see TSDF_LAYER_COLOR): depth_dev as for integrate_depth,
 * color_dev uint32 [height][width] (r in the low byte, then g, b).  Returns
 * TSDF_ERR_ARG for a map of another layer.  Async on cuda_stream.
 */
tsdf_status integrate_color(tsdf_map* map, const float* depth_dev, const uint32_t* color_dev,
                            const tsdf_pinhole* intr, const double T_world_cam[16],
                            void* cuda_stream);

/*
 * integrate_batch — integrate n frames (any mix of sensors, sizes and maps)
 * in sub-batches of up to 32 frames, each one allocation launch and one
 * integration launch; with more than 32 frames the allocation of a
 * sub-batch overlaps the integration of the previous one (on an internal
 * stream of the first map, joined back to cuda_stream).  The result equals
 * integrating the frames one by one in array order (bit for bit with FP32
 * storage; with FP16 storage a voxel is rounded to FP16 once per sub-batch
 * instead of once per frame).  All maps must have been created on the
 * current device; at most 16 distinct maps and 65,536 frames per call.
 */
tsdf_status integrate_batch(tsdf_map* const* maps, int32_t n_maps, const tsdf_frame_desc* frames,
                            int32_t n, void* cuda_stream);

/*
 * integrate_batch_host — integrate_batch for images in HOST memory: each
 * frame's depth_dev (and color_dev) points to host memory, pinned for the
 * copies to overlap the GPU work.  staging_dev (a caller-owned device
 * buffer, 256-byte aligned) is cut into as many slots of one sub-batch's
 * images (each image rounded up to 256 bytes) as fit, 2 to 4; the images of
 * sub-batch b are copied into slot b % slots on an internal copy stream of
 * the first map while earlier sub-batches integrate (contiguous host images
 * of a sub-batch are copied at once).  staging_bytes must hold two slots;
 * TSDF_ERR_ARG otherwise.  Same result as integrate_batch.  The host images
 * must stay valid until the stream passes the call.
 */
tsdf_status integrate_batch_host(tsdf_map* const* maps, int32_t n_maps, const tsdf_frame_desc* frames,
                                 int32_t n, void* staging_dev, int64_t staging_bytes, void* cuda_stream);

/*
 * stage_frames — enqueue n host-to-device copies on cuda_stream: bytes[i]
 * bytes from host src_host[i] (pinned for the copy to be asynchronous) to
 * device dst_dev[i].  A staging helper for callers that place images
 * themselves (a serving loop with its own device ring), one call per batch
 * instead of one per image.  The three arrays are host memory read during
 * the call; the images must stay valid, and the destinations unused, until
 * the stream passes the copies.  TSDF_ERR_ARG for n < 0, a null array, a
 * null pointer or a negative size (nothing is enqueued then); a failed copy
 * returns TSDF_ERR_CUDA after the copies before it were enqueued.
 */
tsdf_status stage_frames(const void* const* src_host, void* const* dst_dev, const int64_t* bytes, int32_t n,
                         void* cuda_stream);

/*
 * query_voxels — TSDF value at n points (float32 [n][3], layer frame,
 * metres): the voxel containing each point, looked up in the block hash.
 * Writes dist_dev[n] and weight_dev[n]; unallocated or unobserved voxels
 * give weight 0 and distance 0.  TSDF_ERR_ARG for a colour map (use
 * query_color).  Async on cuda_stream.
 */
tsdf_status query_voxels(const tsdf_map* map, const float* pts_dev, int64_t n, float* dist_dev,
                         float* weight_dev, void* cuda_stream);

/*
 * query_color — colour at n points of a colour map: rgb_dev float32 [n][3]
 * (r, g, b in 0..255) and weight_dev[n] (colour updates, capped); zeros for
 * unallocated or uncoloured voxels.  TSDF_ERR_ARG for a map of another
 * layer.  Async on cuda_stream.
 */
tsdf_status query_color(const tsdf_map* map, const float* pts_dev, int64_t n, float* rgb_dev,
                        float* weight_dev, void* cuda_stream);

/* map_sync — wait for all work the library enqueued for this map and return
 * its sticky device status (TSDF_OK, TSDF_ERR_CAPACITY or TSDF_ERR_TIMEOUT). */
tsdf_status map_sync(tsdf_map* map);

/* map_num_blocks — number of allocated blocks (synchronises the map). */
tsdf_status map_num_blocks(const tsdf_map* map, int64_t* out);

/* map_stats — counters since creation or the last map_reset (synchronises):
 * out[0] blocks allocated, out[1] voxel updates (voxel, frame pairs that
 * passed the update test), out[2] frames integrated, out[3] sticky device
 * status bits, out[4] block visits (blocks listed by integration launches,
 * summed over launches), out[5] integration launches, out[6] band segments
 * walked (valid pixels), out[7] block-grid cells emitted by those walks
 * (counting a block once per pixel that meets it); out[6] and out[7] count
 * only while map_walk_stats is enabled; out[8] (block, frame) pairs
 * integrated (each projects the block's 512 voxels into the frame). */
tsdf_status map_stats(const tsdf_map* map, int64_t out[9]);

/* map_walk_stats — diagnostics: while enabled, allocation launches that
 * include this map count band segments and walked block-grid cells into
 * map_stats out[6] and out[7] (off by default: it costs about 5 % of the
 * allocation time). */
tsdf_status map_walk_stats(tsdf_map* map, int32_t enable);

/* map_timing — diagnostics: while enabled, every integrate call on this map
 * (or integrate_batch sub-batch whose first map it is) records CUDA events
 * around its allocation and integration kernels, for up to 4096 calls.
 * Enabling creates the events; call it outside any timed region. */
tsdf_status map_timing(tsdf_map* map, int32_t enable);

/* map_kernel_times — waits for the recorded calls and returns the summed
 * device time of their allocation (out_ms[0]) and integration (out_ms[1])
 * kernels and the number of calls recorded; then clears the record.  A fused
 * launch (TSDF_LAUNCH_FUSED) counts whole as allocation time. */
tsdf_status map_kernel_times(tsdf_map* map, double out_ms[2], int64_t* calls);

/*
 * map_export — copy every allocated block to host memory, sorted by block
 * coordinates (x, then y, then z): keys_host int32 [n][3], dist_host and
 * weight_host float32 [n][512] (either may be NULL).  n must equal the block
 * count; returns TSDF_ERR_ARG otherwise.  For a colour map the distances are
 * 0 and the weights are the colour weights.  Synchronises.
 */
tsdf_status map_export(const tsdf_map* map, int32_t* keys_host, float* dist_host,
                       float* weight_host, int64_t n);

/* map_export_color — as map_export for a colour map: keys_host int32 [n][3],
 * rgb_host float32 [n][512][3], weight_host float32 [n][512] (either may be
 * NULL).  TSDF_ERR_ARG for a map of another layer or a wrong n. */
tsdf_status map_export_color(const tsdf_map* map, int32_t* keys_host, float* rgb_host,
                             float* weight_host, int64_t n);

/*
 * map_decay_occupancy — one decay step of an occupancy layer (Sec. V-E: the
 * dynamic part of a scene, kept in its own occupancy layer, fades over
 * time; the paper gives no rule): every allocated voxel's log-odds moves
 * toward 0 (probability 1/2), occupied values (> 0) by decay_occ, free
 * values (< 0) by decay_free, neither crossing 0.  Blocks stay allocated.
 * TSDF_ERR_ARG for another layer or a negative or non-finite step.  Async
 * on cuda_stream.
 */
tsdf_status map_decay_occupancy(tsdf_map* map, float decay_occ, float decay_free,
                                void* cuda_stream);

/*
 * map_import — write n blocks into the map from host memory: keys_host
 * int32 [n][3] block coordinates (each in (-2^20, 2^20), no duplicates),
 * dist_host and weight_host float32 [n][512] (voxel x + 8 y + 64 z; for an
 * occupancy map dist is the log-odds and weight_host may be NULL).  Missing
 * blocks are allocated, present ones overwritten; every written block
 * counts as changed for the next map_esdf_update.  Values are stored in the
 * map's storage (FP16 and FIXED16 round D / tau and W).  Not for colour maps.
 * Synchronises; uses temporary device memory.
 */
tsdf_status map_import(tsdf_map* map, const int32_t* keys_host, const float* dist_host,
                       const float* weight_host, int64_t n);

/* ESDF parameters: site_eps (m): observed voxels with |D| <= site_eps are
 * sites; min_weight: voxels with W >= min_weight are observed; max_dist_vox
 * (1..255): distances are propagated up to this many voxels.  Defaults
 * (NULL): one voxel, 1e-4, 64. */
typedef struct {
  float site_eps;
  float min_weight;
  int32_t max_dist_vox;
} tsdf_esdf_opts;

/*
 * map_esdf_update — bring the map's ESDF layer (Sec. IV-C) up to date with
 * the TSDF blocks changed since the previous call (integrated or imported).
 * Each ESDF voxel is unknown or observed; an observed voxel may be a site and
 * may hold a parent, the offset to the site it is closest to as found by the
 * propagation.  Stages, in order: mark sites in the changed blocks (a voxel
 * that stops being a site, becomes observed or changes sides loses its
 * parent); clear, in blocks within ceil(max_dist / 8) + 1 blocks of one that
 * lost a site, every parent that is no longer a site; then repeat until no
 * block changes: six in-block sweeps (+x, -x, +y, -y, +z, -z) of the update
 * set, and a face exchange (faces -x, +x, -y, +y, -z, +z) in which the
 * update set and its face neighbours take, on their faces, a shorter parent
 * from the adjacent voxel across the face, all reading the states before the
 * exchange.  A parent is taken only if strictly shorter and within
 * max_dist.  The first call allocates the layer (8 KiB per pool block) and
 * fixes the parameters; later calls must pass the same ones.  TSDF maps (any
 * storage) and occupancy maps.  On an occupancy map (Sec. IV-C: an occupancy
 * voxel is a site if it is adjacent to free voxels) a voxel with log-odds
 * l > 0 is occupied (inside), l < 0 free, l = 0 unknown; a site is an
 * occupied voxel with a free voxel among its six face neighbours (a voxel of
 * a missing block is unknown); site_eps and min_weight are not used; the
 * blocks marked are the changed ones and their face neighbours, and a
 * map_decay_occupancy call counts as a change of every block it alters.
 * Enqueued on cuda_stream; waits for the stream after every four iterations
 * to test for convergence.
 */
tsdf_status map_esdf_update(tsdf_map* map, const tsdf_esdf_opts* opts, void* cuda_stream);

/* map_esdf_export — ESDF voxel states of every block, sorted like
 * map_export: keys_host int32 [n][3], states_host uint32 [n][512] (may be
 * NULL).  State word: parent offset x, y, z as 9-bit two's complement in
 * bits 0-8, 9-17, 18-26; bit 27 observed, bit 28 site, bit 29 has a parent,
 * bit 30 inside (D < 0).  TSDF_ERR_ARG before the first update or for a
 * wrong n.  Synchronises. */
tsdf_status map_esdf_export(const tsdf_map* map, int32_t* keys_host, uint32_t* states_host, int64_t n);

/* map_esdf_query — signed Euclidean distance (m) at n points (float32
 * [n][3], device): the voxel's parent offset length times the voxel size,
 * negative inside; +-max_dist voxels for an observed voxel without a parent;
 * NaN for an unknown voxel or a point in no block.  Async on cuda_stream. */
tsdf_status map_esdf_query(const tsdf_map* map, const float* pts_dev, int64_t n, float* dist_dev,
                           void* cuda_stream);

/* map_esdf_stats — totals since the layer was allocated or the map reset:
 * out[0] lowering iterations, out[1] blocks swept, out[2] blocks in face
 * exchanges, out[3] voxels whose parent was cleared.  Synchronises. */
tsdf_status map_esdf_stats(const tsdf_map* map, int64_t out[4]);

/*
 * map_mesh — marching-cubes triangles of the map's TSDF (Sec. IV-B: updated
 * blocks are meshed with a parallel Marching Cubes).  A cube joins the
 * voxel centres g .. g + (1, 1, 1) and belongs to the block of g; it is
 * meshed if its eight voxels exist and have W >= min_weight.  A corner is
 * inside if D < 0; a vertex sits on each edge whose ends differ, at
 * t = D_lo / (D_lo - D_hi) from the lower end.  Faces with two diagonal
 * inside corners keep those corners apart, so neighbouring cubes join
 * without gaps; triangles face the outside (increasing D).  changed_only:
 * only the blocks changed since the previous call and the blocks whose
 * cubes reach into them, else every block.  Output (device): tri_pos_dev
 * float32 [cap][3][3] vertex positions (m); tri_keys_dev int32 [cap][3][4]
 * (may be NULL) the global voxel index of each vertex's lower edge end and
 * the edge axis; tri_cube_dev int32 [cap][3] (may be NULL) the cube's voxel
 * index.  Triangle order is unspecified.  *n_tris = triangles produced;
 * TSDF_ERR_CAPACITY if more than cap (the first cap are written).  TSDF
 * maps only.  Synchronises cuda_stream.
 */
tsdf_status map_mesh(tsdf_map* map, float min_weight, int32_t changed_only, float* tri_pos_dev,
                     int32_t* tri_keys_dev, int32_t* tri_cube_dev, int64_t cap, int64_t* n_tris,
                     void* cuda_stream);

/* map_wait_test — test hook for the bounded wait of TSDF_LAUNCH_FUSED:
 * while extra_ctas > 0, the map's fused launches wait at their grid-wide
 * barrier for extra_ctas more CTAs than they have, so the wait runs out
 * after about a second, the launch skips its integration and the map
 * reports TSDF_ERR_TIMEOUT (cleared by map_reset).  0 restores normal
 * operation.  TSDF_ERR_ARG for a negative count. */
tsdf_status map_wait_test(tsdf_map* map, int32_t extra_ctas);

/* map_reset — drop every block (keeps the allocation), enqueued on
 * cuda_stream; clears the sticky status. */
tsdf_status map_reset(tsdf_map* map, void* cuda_stream);

/* map_destroy — free the map's device memory (synchronises first). */
tsdf_status map_destroy(tsdf_map* map);

/*
 * Allocation-free integration.  The paper has no counterpart: this entry
 * point is for callers that cannot allocate GPU memory when they integrate,
 * because the device allocator belongs to another framework that owns all of
 * the GPU's memory, or because a real-time loop forbids allocation once it
 * has started.  It integrates one pinhole frame exactly like
 * integrate_depth into FP32 map storage that the caller owns, described by
 * tsdf_map_buffers:
 *   keys        uint64 [hash_capacity], every byte 0xFF before first use
 *   vals        int32  [hash_capacity], every byte 0xFF before first use
 *   mask        uint32 [hash_capacity], zero before first use
 *   pool        {float D, float W} [max_blocks][512], any initial contents
 *   block_keys  uint64 [max_blocks]: key of each pool block (written)
 *   counters    uint64 [TSDF_NUM_COUNTERS], zero before first use:
 *               [0] blocks allocated (pool blocks 0 .. min([0], max_blocks) - 1
 *               are in use), [1] voxel updates, [2] status bits (nonzero =
 *               capacity exceeded), [3] block visits, [4] integration
 *               launches, [5] and [6] unused (left as they are), [7] (block,
 *               frame) pairs integrated
 * hash_capacity is a power of two >= 2 * max_blocks.  A block key packs
 * the coordinates plus TSDF_KEY_BIAS into TSDF_KEY_BITS-bit fields:
 * (x + 2^20) | (y + 2^20) << 21 | (z + 2^20) << 42.  Between calls the
 * storage must not be modified.
 *
 * The per-call work list lives in a fixed array of device memory inside the
 * library, reserved on every GPU that loads the library until the process
 * exits: 4 * (TSDF_STATIC_MAX_BLOCKS + 4) bytes.  max_blocks above
 * TSDF_STATIC_MAX_BLOCKS is refused with TSDF_ERR_CAPACITY; other bad
 * arguments give TSDF_ERR_ARG.  The call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.  Its first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call
 * shares the one array and clears its control words before use, so calls
 * whose work overlaps on the GPU (different streams or threads) race and
 * must be serialised by the caller.
 */
#define TSDF_NUM_COUNTERS 8
#define TSDF_KEY_BITS 21
#define TSDF_KEY_BIAS (1 << 20)
#define TSDF_STATIC_MAX_BLOCKS (1 << 16)

typedef struct {
  unsigned long long* keys;
  int32_t* vals;
  uint32_t* mask;
  void* pool;
  unsigned long long* block_keys;
  unsigned long long* counters;
  int64_t hash_capacity;
  int64_t max_blocks;
} tsdf_map_buffers;

tsdf_status integrate_depth_static(const tsdf_map_buffers* buf, float voxel_size,
                                   int32_t truncation_voxels, float max_weight,
                                   const float* depth_dev, const tsdf_pinhole* intr,
                                   const double T_world_cam[16], void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_TSDF_H_ */
