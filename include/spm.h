/*
 * spm.h -- C ABI of the GB300 shortest-path-map (SPM) library.
 *
 * A shortest-path map (arxiv 1805.08500, Sec. 3 "Multi-Source Shortest Path
 * Maps") stores, for every pixel of a polygonal 2D scene, the geodesic
 * distance lambda*(p) to the closest source and the parent generator: the
 * next point of that shortest path, which is a point source, a segment-source
 * endpoint, a segment-source interior foot (Sec. 4 "Segment Sources") or an
 * obstacle vertex. The paper builds it by rasterising clipped cones in OpenGL;
 * this library computes the same field with CUDA kernels for sm_103a.
 *
 * Conventions shared by every call:
 *   - World [0, world_w) x [0, world_h) in integer world units; a grid of
 *     grid_w x grid_h pixels; pixel (i, j) samples its centre
 *     ((i + 0.5) * world_w / grid_w, (j + 0.5) * world_h / grid_h)
 *     (Sec. 6: points are approximated by pixel centres).
 *   - Output planes are row-major, index j * grid_w + i: dist[] (float32)
 *     and parent[] (int32). Unreached or non-free pixels (inside an
 *     obstacle's open interior) get dist = +inf, parent = -1 (the paper's
 *     alpha = 0 "not reached", Sec. 3.1).
 *   - Generator ids: point sources 0..n_points-1; then per segment source k
 *     three ids: endpoint A, endpoint B, interior; then obstacle vertices that
 *     are convex corners of the union of obstacles, polygon-major in input
 *     order, first occurrence of a position kept. Sources are their own parent
 *     (Sec. 3.1, ParentId). Ties between equal distances go to the smaller id.
 *   - Obstacles are convex polygons (3..16 vertices, integer coordinates, any
 *     orientation). Free space is the complement of the union of their open
 *     interiors: touching or grazing a boundary is allowed. Polygons may
 *     overlap (e.g. maze walls); they may not touch at a single point only.
 *   - Predicates run on an integer lattice of scale S (a power of two with
 *     every pixel centre on the lattice and S * scene span <= 32767), so
 *     visibility and cone tests are exact integer arithmetic. Sources are
 *     snapped to that lattice (round to nearest even) for visibility only;
 *     distances use the unsnapped coordinates.
 *
 * Ownership and errors: every call returns an spm_status; no exception or
 * C++ object crosses this boundary. The library owns spm_scene objects;
 * device output buffers passed to spm_compute* stay owned by the caller.
 * Device-side failures (iteration caps, capacity overflows) are latched in a
 * status word that spm_scene_sync() returns. A scene is bound to the CUDA
 * device that was current at creation; call it with that device current.
 */
#ifndef SPM_GB300_H
#define SPM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPM_OK = 0,
    SPM_ERR_INVALID_ARG = 1,   /* null pointer, bad size, wrong device        */
    SPM_ERR_BAD_GEOMETRY = 2,  /* non-convex polygon, source not free, ...    */
    SPM_ERR_OOM = 3,           /* device or host allocation failed           */
    SPM_ERR_CUDA = 4,          /* a CUDA runtime call failed                 */
    SPM_ERR_NOT_CONVERGED = 5, /* vertex-cost fixpoint hit its round cap     */
    SPM_ERR_TIMEOUT = 6,       /* reserved: no kernel of this library waits on
                                  another, so no call returns it              */
    SPM_ERR_CAPACITY = 7       /* a fixed-size device buffer overflowed      */
} spm_status;

typedef struct spm_scene spm_scene;

/* Scene description. All pointers are HOST memory, read during the call and
 * copied; the caller may free them afterwards. */
typedef struct {
    int32_t world_w, world_h;    /* world size in integer units (> 0)        */
    int32_t grid_w, grid_h;      /* pixel grid (> 0)                         */
    int32_t n_polys;             /* number of convex obstacle polygons       */
    const int32_t *poly_offsets; /* n_polys + 1 prefix offsets into vertices */
    const int32_t *poly_xy;      /* 2 * poly_offsets[n_polys] interleaved x,y */
    int32_t n_points;            /* point sources                            */
    const float *point_xy;       /* 2 * n_points                             */
    int32_t n_segments;          /* segment sources (Sec. 4)                 */
    const float *seg_xyxy;       /* 4 * n_segments: ax, ay, bx, by           */
} spm_scene_desc;

/* Validates and prepares a scene (arxiv 1805.08500 Sec. 3.1: the DataArray of
 * sources and obstacle vertices) and allocates every device buffer the
 * compute calls need, on the current device. Rejects with
 * SPM_ERR_BAD_GEOMETRY: a polygon that is not strictly convex or has more
 * than 16 vertices, a source not strictly outside every closed obstacle or
 * outside the world, a zero-length segment or one touching an obstacle, two
 * obstacles touching at one point, a scene too large for the exact lattice.
 * On success *out owns the scene; release it with spm_scene_destroy. */
spm_status spm_scene_create(const spm_scene_desc *desc, spm_scene **out);

/* Frees the scene and its device buffers (synchronises its device first). */
void spm_scene_destroy(spm_scene *scene);

/* Moves the sources (same counts as at creation; host arrays, may be NULL
 * when the count is 0) and re-validates them (Sec. 3.1: sources are the
 * Source entries of the DataArray). The next spm_compute uses them. */
spm_status spm_scene_update_sources(spm_scene *scene, const float *point_xy,
                                    const float *seg_xyxy);

/* Moves the sources from DEVICE arrays, stream-ordered on `stream` (a
 * cudaStream_t, NULL = legacy default stream): the dynamically changing maps
 * of Sec. 6, where sources move every frame and the map is recomputed with no
 * host round trip. point_xy_dev: 2 * n_points floats (x, y); seg_xyxy_dev:
 * 4 * n_segments floats (ax, ay, bx, by), both world units, caller-owned,
 * read by the kernel when it runs (keep them alive and unchanged until then);
 * either may be NULL when its count is 0. A kernel snaps and validates them
 * exactly as spm_scene_update_sources does and then commits all of them, or,
 * when any source is invalid (non-finite, outside the world, not strictly
 * outside every obstacle, a zero-length segment, a segment touching an
 * obstacle), none: the scene keeps its previous sources and the next
 * spm_scene_sync returns SPM_ERR_BAD_GEOMETRY. The next spm_compute on the
 * same stream uses the new sources. Allocates nothing and may be captured in
 * a CUDA graph. Returns SPM_ERR_INVALID_ARG for a null scene or a null array
 * with a non-zero count, SPM_ERR_CUDA when the launch fails. */
spm_status spm_scene_update_sources_device(spm_scene *scene, void *stream,
                                           const float *point_xy_dev,
                                           const float *seg_xyxy_dev);

/* Computes the shortest-path map (Sec. 3: vertex costs relaxed to a fixpoint,
 * then every pixel takes the minimum over visible generators of
 * cost(g) + |p - g|, Procedures 1-4; segment interiors use the perpendicular
 * foot, Sec. 4). Asynchronous on `stream` (a cudaStream_t, NULL = legacy
 * default stream). dist_dev / parent_dev: caller-owned DEVICE buffers of
 * grid_w * grid_h elements, row-major. Allocates nothing. Device-side errors
 * surface through spm_scene_sync. */
spm_status spm_compute(spm_scene *scene, void *stream, float *dist_dev,
                       int32_t *parent_dev);

/* Row slab of the same map, for splitting one scene over several GPUs (no
 * counterpart in the paper; each GPU computes its own slab, and no data is
 * exchanged). Runs the whole vertex phase and culling, then the pixel pass
 * for grid rows [row0, row1) only: row0 and row1 must be multiples of the
 * scene's tile size (spm_scene_info()[7]) or row1 == grid_h, else
 * SPM_ERR_INVALID_ARG. dist_dev / parent_dev are the full-grid buffers of
 * spm_compute; only the slab's rows are written, with the values
 * spm_compute writes there. Queries (spm_query_parent, spm_extract_path)
 * need a whole-grid spm_compute. Asynchronous; allocates nothing. */
spm_status spm_compute_rows(spm_scene *scene, void *stream, int32_t row0, int32_t row1,
                            float *dist_dev, int32_t *parent_dev);

/* The same map by the paper's own schedule (Sec. 3.1, Procedures 1-4): one
 * generator at a time, in order of cost, over every pixel -- the search for
 * the least-cost unexpanded generator (Procedure 1), the update of the
 * obstacle vertices it sees (Procedure 4) and a depth-tested pass over all
 * pixels with exact visibility in place of the shadow stencil (Procedures
 * 2-3), in one cooperative kernel with a grid barrier per generator. An A/B
 * baseline for spm_compute: like the paper it has no shadow cones and no
 * visibility-graph tangency filter, so distances agree with spm_compute to
 * FP32 rounding and parents agree except at (near-)ties. dist_dev /
 * parent_dev: caller-owned device buffers as for spm_compute (they also
 * serve as the depth buffer). Uses the scene's vertex-phase scratch, so do
 * not run it concurrently with another compute of the same scene; leaves
 * the generator table of the last spm_compute (and so the queries)
 * untouched. Asynchronous; allocates nothing. SPM_ERR_CAPACITY above 65536
 * generators, SPM_ERR_CUDA when the cooperative launch fails. */
spm_status spm_compute_sequential(spm_scene *scene, void *stream, float *dist_dev,
                                  int32_t *parent_dev);

/* spm_compute on HOST buffers, complete when it returns (synchronous on
 * `stream`). For callers that keep the field on the host. Page-locked
 * buffers (cudaHostAlloc, torch pin_memory) receive the map directly from the
 * pixel pass. Pageable ones receive it through device staging planes,
 * allocated on the first call, in row slabs copied while the next slab
 * computes. The scene keeps no pointer to the host buffers: the caller may
 * unpin or free them once the call returns. After a compute into page-locked
 * buffers the field queries (spm_query_parent, spm_query_exact,
 * spm_extract_path) have no field to read and return SPM_ERR_INVALID_ARG
 * until the next device compute; after one into pageable buffers they read
 * the staging planes. */
spm_status spm_compute_host(spm_scene *scene, void *stream, float *dist_host,
                            int32_t *parent_host);

/* Computes n independent scenes in one batched, persistent launch sequence
 * (all scenes' vertex phases, then one persistent pixel kernel over every
 * scene's tiles, largest first). dist[k] / parent[k] are caller-owned device
 * buffers of scene k's grid. All scenes must live on the current device.
 * Convenience form of spm_batch_create + spm_batch_compute +
 * spm_batch_destroy: it allocates the batch descriptors and waits for the
 * stream before returning; keep an spm_batch for repeated calls. */
spm_status spm_compute_batched(spm_scene *const *scenes, int32_t n, void *stream,
                               float *const *dist, int32_t *const *parent);

/* A batch: n scenes computed together by one launch sequence (vertex phase of
 * every scene in batched kernels, then one persistent pixel kernel over all
 * scenes' tiles, largest scenes first), captured once into a CUDA graph and
 * replayed by spm_batch_compute. dist[k] / parent[k] are caller-owned device
 * buffers of scene k's grid, fixed for the batch's lifetime. Creation
 * allocates the batch's device descriptors; compute allocates nothing. The
 * scenes must outlive the batch; culling and tile settings are read at
 * creation. A scene in the geometric flood mode (flood_mode 3) floods only
 * its sources in the batch, over the lists of its obstacle vertices built
 * once (at creation, or again by a compute whose tuning replaced them). */
typedef struct spm_batch spm_batch;
spm_status spm_batch_create(spm_scene *const *scenes, int32_t n, float *const *dist,
                            int32_t *const *parent, spm_batch **out);
spm_status spm_batch_compute(spm_batch *batch, void *stream);
void spm_batch_destroy(spm_batch *batch);

/* Device time of the last spm_batch_compute, in milliseconds, from events
 * recorded inside its launch sequence (event nodes of its CUDA graph):
 * vertex_ms = every scene's vertex phase and candidate lists, pixel_ms = the
 * persistent pixel kernel. Waits for that compute. */
spm_status spm_batch_phase_ms(spm_batch *batch, float *vertex_ms, float *pixel_ms);

/* Waits for the scene's last work on `stream` and returns the first latched
 * device-side or CUDA error (SPM_OK if none), clearing it. */
spm_status spm_scene_sync(spm_scene *scene, void *stream);

/* O(1) point location (Sec. 1: "point localization is reduced to a simple
 * constant time grid buffer mapping"): pixel containing world point (x, y)
 * in the last computed field; writes its parent id and distance. Synchronous
 * (reads one pixel back). SPM_ERR_INVALID_ARG if (x, y) is outside the world
 * or nothing was computed yet. */
spm_status spm_query_parent(spm_scene *scene, float x, float y, int32_t *parent,
                            float *dist);

/* Exact point query (Sec. 6, Discussion: a point on a region border may take
 * a parent up to half a pixel's diagonal off, and comparing the neighbouring
 * parents at the point itself removes the error). The parents of the 3 x 3
 * pixels around (x, y) in the last whole-grid compute are evaluated at the
 * lattice point nearest (x, y) with the exact visibility and cone tests and
 * FP64 distances at (x, y) itself; writes the closest (ties: smaller id) and
 * its distance, -1 / +inf when none is valid there. Synchronous (one small
 * kernel on the compute's stream). SPM_ERR_INVALID_ARG when (x, y) is outside
 * the world or nothing was computed yet. */
spm_status spm_query_exact(spm_scene *scene, float x, float y, int32_t *parent,
                           float *dist);

/* Shortest path from world point (x, y) back to its source (Sec. 1: the path
 * is retrieved by following parents, linear in its number of vertices).
 * Writes the polyline to out_xy (2 floats per point, starting at (x, y),
 * ending at the source point or the perpendicular foot on a segment source)
 * and the point count to *n. SPM_ERR_CAPACITY if more than cap points. */
spm_status spm_extract_path(spm_scene *scene, float x, float y, float *out_xy,
                            int32_t cap, int32_t *n);

/* Generator table after the last spm_compute (synchronous copy to the host
 * arrays, each of length spm_scene_info()[0]; any pointer may be NULL):
 * kind (0 point, 1 segment A, 2 segment B, 3 segment interior, 4 obstacle
 * vertex), lattice position (2 per generator), FP64 cost and parent id.
 * The visibility graph keeps only links tangent to the obstacles at both
 * ends (a shortest path bends around a vertex, Sec. 3.1), so an obstacle
 * vertex that no tangent link reaches at its geodesic distance -- one reached
 * only head-on, whose shadow cone is empty and which is never a parent --
 * reports a cost above that distance (or +inf). Every vertex that can be a
 * parent reports its exact geodesic distance; the map is unaffected. */
spm_status spm_scene_generators(spm_scene *scene, int32_t *kind, int32_t *lattice_xy,
                                double *cost, int32_t *parent);

/* info must hold 11 entries: [0] generators, [1] sources (incl. 3 per
 * segment), [2] obstacle-vertex generators, [3] lattice scale S, [4]
 * polygons, [5] vertex-phase rounds of the last compute (after sync), [6]
 * visibility-graph edges of the last compute (after sync), [7] tile size in
 * pixels, [8] 1 if the last compute used flooded per-tile candidate lists
 * (after sync), [9] flood_mode, [10] kernels one spm_compute launches with
 * the current settings. */
spm_status spm_scene_info(spm_scene *scene, int64_t *info);

/* Differentiable form. Forward: loss = mean over n agents (pixel indices,
 * int32 (i, j) pairs in DEVICE memory) of the field value in dist_dev (an
 * spm_compute result of this scene); writes the scalar to loss_dev (device
 * float). Agents on unreached pixels count as 0. When tape_dev is not NULL,
 * the forward also records on it what the backward needs: each agent's
 * contribution to d loss / d sources, from its root link -- the last leg of
 * its parent chain in parent_dev (Sec. 3.1 ParentId chain) and the current
 * source positions. Call it on the compute's stream, before the next compute
 * of this scene, so that the chain is the one of that compute's generator
 * table. tape_dev: caller-owned DEVICE memory of spm_agents_tape_bytes(n)
 * bytes, 16-byte aligned. Asynchronous on `stream`; allocates nothing. */
spm_status spm_agents_forward(spm_scene *scene, void *stream, const int32_t *agents_dev,
                              int32_t n, const float *dist_dev, const int32_t *parent_dev,
                              float *loss_dev, void *tape_dev);

/* Bytes of the tape spm_agents_forward records for n agents (0 for n < 0). */
int64_t spm_agents_tape_bytes(int32_t n);

/* Backward: d loss / d point sources (grad_points_dev, 2 * n_points floats)
 * and d loss / d segment endpoints (grad_segs_dev, 4 * n_segments floats)
 * from a tape recorded by spm_agents_forward for the same n agents: the mean
 * of the agents' root-link gradients, summed in a fixed order (the result is
 * deterministic). Reads the tape and the scene's source counts only, so a
 * later compute or source move of the scene does not change it, and several
 * tapes of one scene may be held at once. Asynchronous on `stream`. */
spm_status spm_agents_backward(spm_scene *scene, void *stream, const void *tape_dev,
                               int32_t n, float *grad_points_dev, float *grad_segs_dev);

/* Allocation-free variant of spm_agents_backward. The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory while they run, such as a per-frame agent-steering loop in a
 * game or crowd simulation, where a cudaMalloc can stall the frame, or code
 * living inside a framework whose memory pool owns the device and forbids raw
 * cudaMalloc calls.
 *
 * It computes the same gradient as spm_agents_forward (with a tape) followed
 * by spm_agents_backward, for n agents (int32 (i, j) pixel pairs, DEVICE
 * memory) on the parent field parent_dev of the last spm_compute of this
 * scene (call it before the next compute or source move), writing
 * grad_points_dev (2 * n_points floats) and grad_segs_dev (4 * n_segments
 * floats), asynchronously on `stream`. It calls no allocating function: its
 * scratch is one fixed array inside the library (about 3.8 MB, held on every
 * GPU that loads the library until the process exits), sized for at most
 * SPM_NOALLOC_MAX_AGENTS agents and SPM_NOALLOC_MAX_GENERATORS generators;
 * larger inputs return SPM_ERR_CAPACITY. The first call on each device looks
 * up the array's device address (once, with that device current); make that
 * first call before any stream capture. All calls share the one array, so
 * calls whose kernels overlap on the GPU (different streams, no ordering)
 * race and give wrong gradients; calls on one stream are safe. */
#define SPM_NOALLOC_MAX_AGENTS 131072
#define SPM_NOALLOC_MAX_GENERATORS 65536
spm_status spm_agents_backward_noalloc(spm_scene *scene, void *stream,
                                       const int32_t *agents_dev, int32_t n,
                                       const int32_t *parent_dev, float *grad_points_dev,
                                       float *grad_segs_dev);

/* Device time of the three phases of the last spm_compute on this scene, in
 * milliseconds, from CUDA events the library records between them on the
 * compute stream (not recorded while the stream is being captured into a
 * CUDA graph): vertex_ms = vertex-cost fixpoint (Sec. 3.1 Procedures 1, 2
 * and 4), cull_ms = the per-tile candidate lists after the vertex phase (the
 * flood; in flood mode 3 it runs beside the vertex phase from the start of
 * the compute, so only the part that outlasts the vertex phase counts; 0
 * when the scene scans every generator), pixel_ms = the pixel kernel
 * (Procedure 3). Waits for the compute. */
spm_status spm_scene_phase_ms(spm_scene *scene, float *vertex_ms, float *cull_ms,
                              float *pixel_ms);

/* Tuning of the pixel pass's culling, per scene.
 * flood_mode: 0 = automatic (flood the per-tile candidate lists when the
 *   visibility graph among generators is sparse -- below 1% of all pairs,
 *   as in mazes -- otherwise let every tile scan every generator; decided on
 *   the device each compute), 1 = always flood, 2 = never flood, 3 = flood
 *   from geometry alone (every generator's visible tiles, no shadow cone) on
 *   the scene's own side stream, concurrently with the vertex phase; the
 *   pixel pass then applies costs and cones.
 * hidden_chunk: first chunk of lb-ordered candidates whose tiles are tested
 *   for being hidden (32..256; later chunks double).
 * tile: pixel tile side, 16 or 32 (default 16 when a pixel spans 8 world
 *   units or more, else 32): each tile is one CTA of the pixel pass.
 * maps: 1 = the flood keeps each point generator's angular depth map and the
 *   pixel pass decides most pixels' visibility from it (exact bounds; only
 *   the undecided pixels take the exact polygon test), 0 = every pixel takes
 *   the exact test (default). Only with a flood (flood_mode != 2) and when
 *   the maps fit (n_gen x 16 KB <= 256 MB).
 * fixpoint_start: where the vertex fixpoint (Sec. 3.1, Procedures 1 and 4)
 *   starts. A scene with 256 to 6144 obstacle vertices and at most 7168
 *   generators whose graph a single fixpoint kernel takes gets, from
 *   spm_scene_create, a table of the geodesic distances between its obstacle
 *   vertices (obstacles never move; n_vert^2 doubles of device memory). 2 =
 *   start from the shortest-path tree that table gives (four extra kernels
 *   per compute); 1 = start from the sources alone; 0 = automatic (default):
 *   the tree when the scene has the table and its trees are deep (the table
 *   build's deepest search took 32 rounds or more, as in mazes), else the
 *   sources. Every choice reaches the same unique fixpoint, bit for bit; the
 *   tree saves the rounds a start from the sources spends carrying costs
 *   down long chains of links. Ignored by the batched form, which always
 *   starts from the sources. */
typedef struct {
    int32_t flood_mode;
    int32_t hidden_chunk;
    int32_t tile;
    int32_t maps;
    int32_t fixpoint_start;
    int32_t reserved[3];
} spm_tuning;

spm_status spm_scene_get_tuning(const spm_scene *scene, spm_tuning *out);
spm_status spm_scene_set_tuning(spm_scene *scene, const spm_tuning *tuning);

/* Autotuner: times spm_compute on this scene (device events on `stream`,
 * warm-up then the median of 3 runs) for every flood_mode x hidden_chunk x
 * tile x maps combination in {1, 2, 3} x {32, 256} x {16, 32} x {0, 1} (maps
 * only with a flood), keeps the fastest and
 * writes it to *chosen (may be NULL). Synchronous. Allocates the scene's
 * output staging planes on first use; call it at set-up, not inside a
 * captured stream. */
spm_status spm_scene_autotune(spm_scene *scene, void *stream, spm_tuning *chosen);

/* Static text for a status code. */
const char *spm_status_string(spm_status status);

/* Last error message recorded for this scene (or for creation failures when
 * scene is NULL); valid until the next call on the same thread. */
const char *spm_last_error(const spm_scene *scene);

/* Test hook for the failure paths (no counterpart in the paper): the n-th
 * next device allocation of the library fails (n = 0: the next one), as if
 * the device were out of memory; n < 0 switches it off (the default). The
 * call that meets the failure returns SPM_ERR_OOM and frees what it had
 * allocated. Process-wide; has no effect unless called. */
void spm_debug_fail_alloc_after(int32_t n);

/* Test hook for the fixpoint's failure path (no counterpart in the paper):
 * n > 0 caps the vertex fixpoint at n rounds in every later compute (and
 * batch created later), so that a scene needing more rounds reports
 * SPM_ERR_NOT_CONVERGED through spm_scene_sync; n <= 0 restores the default
 * cap of 4 rounds per generator plus 64. The kernel stops at the cap and
 * returns normally; the scene stays usable. Process-wide; no effect unless
 * called. */
void spm_debug_set_round_cap(int32_t n);

/* Test hook (no counterpart in the paper): on != 0 makes every later
 * compute solve the vertex fixpoint of a graph the single-CTA kernel does not
 * take, and every batch created later solve all its scenes' fixpoints, with
 * the many-CTA kernel (synchronous rounds between grid barriers) instead of
 * the cluster kernel, so that tests can compare the two; on == 0 restores
 * the default choice. Process-wide; no effect unless called. */
void spm_debug_set_many_cta_fixpoint(int32_t on);

#ifdef __cplusplus
}
#endif

#endif /* SPM_GB300_H */
