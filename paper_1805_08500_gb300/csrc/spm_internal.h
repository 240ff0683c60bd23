// spm_internal.h -- data layout shared by the host preparation, the kernels
// and the C ABI of the shortest-path-map library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/spm.h"

namespace spm {

constexpr int kMaxPolyVerts = 16;    // convex polygon vertex limit
constexpr int kAngBins = 2048;       // pseudo-angle bins of a generator's depth map
constexpr int kTile = 32;            // largest pixel tile side (one CTA per tile)
constexpr int kTileSmall = 16;       // small tile side, for coarse grids
constexpr int kPixelThreads = 256;   // 32x32 tiles: 4 pixels per thread; 16x16: 1
constexpr int kCandCap = 1024;       // candidate generators per batch (smem)
constexpr int kBlockCap = 96;        // blocker polygons per chunk (smem)
constexpr int kDedupBits = 8192;     // polygon-id dedup bitmap (smem)
constexpr int kMaxRounds = 1 << 20;  // hard cap on vertex-fixpoint rounds
constexpr int kSeqMaxGen = 1 << 16;  // generators the sequential (paper-schedule) kernel takes
constexpr int kLocBins = 256;        // pseudo-angle bins of an obstacle vertex's local depth map

enum GenKind : int32_t { kPoint = 0, kSegA = 1, kSegB = 2, kSegI = 3, kVert = 4 };
enum ConeType : int32_t { kConeNone = 0, kConeWedge = 1, kConeRay = 2, kConeEmpty = 3 };

// Device status word bits (latched, read by spm_scene_sync).
enum StatusBits : uint32_t {
    kStNotConverged = 1u,
    kStEdgeOverflow = 2u,
    kStTimeout = 4u,
    kStBadInput = 8u,
    kStBadSource = 16u,  // a device-side source update was rejected (table unchanged)
};

// Host-side prepared scene (lattice integers, generator table, bins).
struct HostScene {
    int32_t Wx = 0, Wy = 0, Nx = 0, Ny = 0;
    int32_t S = 1;                     // lattice scale
    // polygons (lattice, CCW)
    std::vector<int32_t> poly_off;     // P + 1
    std::vector<int32_t> poly_v;       // 2 * V (x, y interleaved)
    std::vector<int32_t> poly_box;     // 4 * P (x0, y0, x1, y1)
    // uniform bins of polygon ids over [bin_x0, ..) x [bin_y0, ..)
    int32_t bin_x0 = 0, bin_y0 = 0, bin_size = 1, bin_nx = 1, bin_ny = 1;
    std::vector<int32_t> bin_start;    // nbins + 1
    std::vector<int32_t> bin_items;
    // sources as given (true coordinates)
    std::vector<float> points;         // 2 * n_points
    std::vector<float> segs;           // 4 * n_segs
    // generators
    int32_t n_gen = 0, n_src = 0, n_vert = 0;
    std::vector<int32_t> gen_kind;     // n_gen
    std::vector<int32_t> gen_lat;      // 2 * n_gen lattice position
    std::vector<float> gen_pos;        // 2 * n_gen true position (world units)
    std::vector<int32_t> gen_aux;      // segment index / source index / polygon vertex index
    std::vector<int32_t> gen_wedge;    // 4 * n_gen obstacle wedge (start xy, end xy), CCW
    // segments on the lattice
    std::vector<int32_t> seg_lat;      // 4 * n_segs
};

// Builds a HostScene from the C descriptor; on failure returns a status and
// an explanatory message.
spm_status prepare_scene(const spm_scene_desc &d, HostScene &hs, std::string &err);
// Re-snaps and re-validates sources of an existing HostScene.
spm_status update_sources(HostScene &hs, const float *pts, const float *segs,
                          std::string &err);

// One polygon entry of a bin, packed so a walk needs a single 32-byte load
// per polygon instead of a chain (id -> box -> offset -> vertices).
struct __align__(16) BinRec {
    int4 box;
    int32_t poly, voff, m, pad;
};

// Device pointers of one scene (all allocated at creation).
struct DevScene {
    int32_t Wx, Wy, Nx, Ny, S;
    float hx, hy;                      // pixel size in world units
    int32_t n_poly, n_gen, n_src, n_vert, n_seg;
    // polygons
    const int32_t *poly_off;
    const int2 *poly_v;
    const int4 *poly_box;
    int32_t bin_x0, bin_y0, bin_size, bin_nx, bin_ny;
    const int32_t *bin_start, *bin_items;
    const BinRec *bin_recs;            // parallel to bin_items
    const uint32_t *free_bits;         // free-space mask of pixel centres, free_words words per grid row
    int32_t free_words;
    // local depth map of each obstacle vertex (kLocBins floats, n_vert rows;
    // null when too large): per pseudo-angle bin an upper bound of the
    // squared distance beyond which every ray of the bin has entered an
    // obstacle, from the polygons near the vertex -- a conservative filter
    // of hidden vertex pairs before the exact test
    const float *vert_maps;
    // generators (static part)
    const int32_t *gen_kind;
    const int2 *gen_lat;
    const float2 *gen_pos;
    const int32_t *gen_aux;
    const int4 *gen_wedge;
    const int4 *seg_lat;               // A.x A.y B.x B.y lattice
    const float4 *seg_pos;             // true coordinates
    // vertex phase
    uint32_t *vis_bits;                // n_vert rows x vis_words
    int32_t vis_words;
    // bits of the obstacle-vertex pairs alone, same layout (built once per
    // scene: obstacles never move; null when every compute tests every pair)
    const uint32_t *vis_static;
    // the pair kernel's range: words 0..pair_words-1 of every row, generators
    // u in [pair_u0, pair_u1) (with vis_static: the source columns only)
    int32_t pair_words, pair_u0, pair_u1;
    int32_t *in_start;                 // n_vert + 1 (by target vertex)
    int32_t *in_src;                   // E
    double *in_len;                    // E
    int32_t *out_start;                // n_gen + 1 (by source generator)
    int32_t *out_dst;                  // E
    int32_t *out_fill;                 // n_gen cursors
    // the obstacle-vertex edges, fixed with the obstacles: in-lists with their
    // FP64 lengths and out-lists, CSR over the obstacle vertices; a compute
    // builds the sources' edges and copies these after them (null: every
    // edge is built per compute)
    const int32_t *st_start;           // n_vert + 1
    const int32_t *st_src;             // generator ids, increasing within a row
    const double *st_len;
    const int32_t *st_out_start;       // n_vert + 1 (by obstacle vertex)
    const int32_t *st_out_dst;
    const int32_t *st_out_init;        // n_gen + 1: out_start before the sources' edges are counted
    int64_t edge_cap;
    // warm start of the fixpoint: geodesic distances between obstacle
    // vertices over the kept edges (n_vert x n_vert FP64, row-major by the
    // first vertex; built once per scene, null when the scene has none), the
    // estimates and tree a compute derives from them, and the state the
    // fixpoint kernels start from when `warm` is set
    const double *vtab;
    int32_t warm;                      // this compute starts from vtab's tree (else from the sources alone)
    double *warm_est;                  // n_vert estimated costs
    int32_t *warm_tpar;                // n_vert tree parents (generator ids, -1: none)
    double *warm_tlen;                 // n_vert FP64 lengths of the tree links
    double *warm_cost;                 // n_gen costs along the tree
    int32_t *warm_par;                 // n_gen parents along the tree
    double *cost[2];                   // Jacobi double buffer
    int32_t *par[2];
    int32_t *frontier[2];              // changed-vertex lists, alternating by round
    int32_t *dirtyl[2];                // vertices to pull, alternating by round
    uint32_t *dirty;                   // n_gen bits: vertex already in the dirty list
    int32_t *counters;                 // [0,1] frontier sizes, [2,3] dirty-list sizes
    int32_t sssp_blocks;               // cooperative grid size (CTAs)
    int32_t solo_smem;                 // shared memory the single-CTA fixpoint may use (0: not available)
    int32_t fix_launch;                // fixpoint kernels a compute launches (kFix* bits)
    // finalised generator table (read by the pixel kernel)
    float *gen_costf;                  // n_gen (inf when unreached)
    double *gen_cost;                  // n_gen
    int32_t *gen_par;                  // n_gen
    int4 *gen_cone;                    // c1.x c1.y c2.x c2.y (lattice directions)
    int32_t *gen_ctype;                // ConeType
    uint32_t *status;                  // latched status bits
    int32_t *stats;                    // [0] rounds, [1] edges
    // tiles and their candidate lists (flood)
    int32_t tile;                      // tile side in pixels: 16 or 32
    int32_t tiles_x, tiles_y;
    int32_t use_flood;                 // 0: flood impossible (too many tiles for smem)
    int32_t flood_mode;                // 0 auto (sparse visibility graph), 1 on, 2 off, 3 geometric (concurrent)
    int32_t hidden_chunk;              // first hidden-test chunk in the pixel pass
    int32_t use_maps;                  // keep and use the flood's depth maps (needs gen_maps)
    int32_t *tile_start;               // ntiles + 1 (CSR by tile)
    int32_t *tile_count;               // ntiles (counts, then fill cursors)
    int32_t *tile_items;               // pair_cap generator ids
    int2 *pairs;                       // pair_cap (tile, generator)
    // per-generator angular depth maps kept by the flood for the pixel pass
    // (null when the scene has too many generators for them): kAngBins
    // float2 (upper bound of the squared distance at which every ray of the
    // bin is inside an obstacle, lower bound of the squared distance at which
    // any ray of the bin can first meet one) per generator, and a flag per
    // generator set when its map is complete for this compute
    float2 *gen_maps;
    uint8_t *gen_map_ok;
    int32_t pair_cap;
    int32_t *glob_list;                // generators every tile scans
    int32_t *flood_counts;             // [0] pairs, [1] global list size, [2] overflow, [3] work counter
    // the geometric flood (mode 3) of the obstacle-vertex generators depends
    // on the obstacles alone: its per-tile lists are kept here (CSR), with
    // its global entries at the front of `glob_list`, its depth maps in
    // gen_maps and its flood_counts[0..2] in static_counts, so that a compute
    // floods and sorts only the sources; a tile's candidates are then its
    // static list, its list of source entries and the global list
    int32_t *static_tile_start;        // ntiles + 1 (small-tile sizing)
    int32_t *static_tile_items;        // pair_cap
    int32_t *static_counts;            // 4
    int32_t static_lists;              // the pixel pass reads the static lists as well (this compute)
    int32_t flood_reuse;               // in a batch's copy: flood the sources only, over the static part
    int32_t src_direct;                // in a batch's copy: those sources culled directly (complete maps)
};

// A batch of scenes computed together (device-side descriptor).
struct BatchDev {
    int32_t n;                         // scenes
    const DevScene *scenes;            // n descriptors (device memory)
    // prefix offsets over scenes (n + 1 entries each)
    const long long *pair_off;         // warp tasks of the visibility pairs: n_vert * pair_words
    const int32_t *vert_off;           // obstacle-vertex generators
    const int32_t *gen_off;            // generators
    const int32_t *flood_off;          // generators the batched flood takes per scene (sources only when reusing)
    // pixel pass: scenes in processing order (costliest tiles first)
    const int32_t *order;              // n scene indices
    const int32_t *tile_off;           // n + 1 prefix of tiles in that order
    int32_t total_tiles;
    int32_t *tile_counter;             // persistent-kernel work counter
    float *const *dist;                // n output planes (device pointers)
    int32_t *const *parent;
    // fixpoint over all scenes: (scene, vertex) lists and counters
    int2 *dirtyl[2];
    int2 *frontier[2];
    int32_t *counters;                 // [0,1] frontier sizes, [2,3] dirty sizes, [4] rounds
    int32_t max_rounds;
    int32_t sssp_blocks;
    int32_t flood_smem;                // dynamic shared memory of the batched flood (0: no scene floods)
    int32_t any_maps;                  // some scene keeps depth maps
    // direct culling of the sources of scenes with src_direct (n + 1 prefixes):
    const long long *src_map_off;      // map entries: n_src * kAngBins
    const long long *src_ins_off;      // warp tasks of the map building: n_src * n_poly
    const long long *src_tile_off;     // warp tasks of the tile tests: n_src * tiles
    int32_t walk_tasks;                // (scene, generator) walks of the batched flood
    // vertex fixpoint on resident clusters, one scene at a time
    const int32_t *cl_order;           // n scene indices, most generators first
    int32_t *cl_done;                  // n flags: a cluster took the scene's fixpoint
    int32_t *cl_counter;               // the clusters' work counter
    int32_t cl_grid;                   // CTAs of the clusters' launch (0: no cluster kernel)
    int32_t cl_all;                    // the clusters take every scene: no many-CTA kernel
};

// Kernel launchers (spm_vertex.cu / spm_pixel.cu / spm_grad.cu).
// vertex phase (visibility graph, fixpoint, finalised generator table)
// A second stream for work of the vertex phase that can run beside its
// chain, with the events that fork it from and join it to the chain.
struct VertexSide {
    cudaStream_t st;
    cudaEvent_t fork, join;
};
void launch_vertex_phase(const DevScene &ds, cudaStream_t st, const VertexSide *side = nullptr);
// pixel kernel over the tiles of tile rows [tile_row0, tile_row1)
void launch_pixel_phase(const DevScene &ds, cudaStream_t st, float *dist, int32_t *parent, int tile_row0,
                        int tile_row1);
// flood of the per-tile candidate lists. FloodStatic::kNone floods every
// generator; kBuild (geometric mode) floods the obstacle vertices, keeps
// their lists as the static part, then floods the sources; kReuse restores
// the static part and floods the sources only.
enum class FloodStatic { kNone, kBuild, kReuse };
void launch_flood(const DevScene &ds, cudaStream_t st, FloodStatic how = FloodStatic::kNone);
// visibility bits of the obstacle-vertex pairs into ds.vis_static (once per scene)
void launch_vis_static(const DevScene &ds, cudaStream_t st, uint32_t *vis_static);
// free-space mask of the pixel centres (once per scene)
void launch_free_mask(const DevScene &ds, cudaStream_t st, uint32_t *bits);
// local depth maps of the obstacle vertices (once per scene)
void launch_vert_maps(const DevScene &ds, cudaStream_t st, float *maps);
// the paper's generator-sequential schedule over the whole map (cooperative launch of `blocks` CTAs)
cudaError_t launch_sequential(const DevScene &ds, cudaStream_t st, float *dist, int32_t *parent, int blocks);
int sequential_grid_blocks();
// validates and commits new source coordinates (device arrays) on `st`
void launch_update_sources(const DevScene &ds, cudaStream_t st, const float *pts, const float *segs);
void launch_vertex_phase_batched(const BatchDev &b, cudaStream_t st);
void launch_pixel_phase_batched(const BatchDev &b, cudaStream_t st);
// src_ins / src_tiles: the totals of b.src_ins_off / b.src_tile_off (host copies)
void launch_flood_batched(const BatchDev &b, cudaStream_t st, long long src_ins, long long src_tiles);
// exact query at lattice point (qx, qy), world (fx, fy), pixel (i, j) of the last field
void launch_query_exact(const DevScene &ds, cudaStream_t st, const int32_t *field_parent, int i, int j, int qx,
                        int qy, double fx, double fy, int32_t *out_par, double *out_dist);
int sssp_batched_grid_blocks();
int fixpoint_round_cap(int n_gen);  // rounds the vertex fixpoint may take (test hook aside: 4 n_gen + 64)
bool flood_possible(int tiles, int polys);
size_t flood_smem_bytes(int tiles, int polys, bool maps);  // dynamic shared memory of one flood CTA
int flood_smem_attr();
// the geometric mode culls the sources directly (complete depth maps, every
// tile tested at once) rather than by the per-generator walk
bool flood_sources_direct(const DevScene &ds);
int sssp_grid_blocks();  // co-resident CTAs for the cooperative fixpoint kernel
int solo_smem_bytes();   // shared memory granted to the single-CTA fixpoint kernel (0 if refused)
bool cluster_smem_ok();  // the cluster fixpoint can run (its shared memory was granted)
int cluster_ctas();      // CTAs of a single scene's cluster fixpoint (16, or 8 where 16 do not fit; 0: unavailable)
// fixpoint kernels of a scene's computes: the single-CTA one, the cluster
// one, and whether one of them surely takes every compute's graph (then the
// many-CTA kernel is not launched)
constexpr int kFixSolo = 1, kFixCluster = 2, kFixSoloSure = 4, kFixClusterSure = 8;
constexpr int kFixClusterFits = 16;  // the cluster kernel takes every compute's graph (batched form)
constexpr int kFixClusterWide = 32;  // the cluster kernel runs on 16 CTAs (else 8)
// from the static in-degrees (scene creation)
int fixpoint_launches(const DevScene &ds, const std::vector<int32_t> &deg);
// FP64 lengths of the static in-lists (ds.st_start / st_src set), into len
void launch_static_lengths(const DevScene &ds, double *len, cudaStream_t st);
// the warm start's geodesic table over the kept obstacle-vertex edges
// (once per scene; ds.st_* set): tab gets n_vert x n_vert doubles
constexpr int kVtabMinVert = 256;   // smaller graphs converge in a few rounds from the sources
constexpr int kVtabMaxVert = 6144;  // the table's size: n_vert^2 doubles (288 MB at the limit)
constexpr int kWarmMaxGen = 7168;   // generators the tree-fold kernel holds in shared memory
constexpr int kWarmMinDepth = 32;   // table-build rounds from which the warm start is the default
bool vtab_possible(const DevScene &ds);
cudaError_t launch_vtab_build(const DevScene &ds, double *tab, int32_t *counter, cudaStream_t st);
int cluster_batched_grid();  // CTAs of the batched cluster fixpoint's launch (0: unavailable)
int count_kernel_launches_vertex();
int count_kernel_launches_pixel();
// differentiable form (spm_grad.cu): the per-agent contributions of the
// root links (slot = first gradient component, val = up to four values), and
// their deterministic two-level reduction into the gradient
constexpr int kGradPartials = 65536;  // partial sums of the reduction (chunks x components)
int grad_chunks(int n_out);
constexpr int kLossPartials = 64;  // partial sums of the loss (scratch doubles)
void launch_agents_forward(const DevScene &ds, cudaStream_t st, const int32_t *agents, int n, const float *dist,
                           float *loss, double *partial);
void launch_agents_contrib(const DevScene &ds, cudaStream_t st, const int32_t *agents, int n,
                           const int32_t *parent, int32_t *root, float2 *lastpt, int32_t *slot, float4 *val);
void launch_agents_reduce(int n_pts, int n_seg, cudaStream_t st, const int32_t *slot, const float4 *val, int n,
                          double *partial, float *grad_pts, float *grad_segs);
void launch_agents_backward(const DevScene &ds, cudaStream_t st, const int32_t *agents, int n,
                            const int32_t *parent, int32_t *root, float2 *lastpt, int32_t *slot,
                            float4 *val, double *partial, float *grad_pts, float *grad_segs);
}  // namespace spm

struct spm_scene;
namespace spm {
const DevScene *scene_dev(const spm_scene *s);
int scene_device(const spm_scene *s);
void scene_set_error(spm_scene *s, const char *msg);

}  // namespace spm
