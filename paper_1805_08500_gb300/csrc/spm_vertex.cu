// spm_vertex.cu -- vertex phase: costs of obstacle-vertex generators.
//
// arxiv 1805.08500 Sec. 3.1 settles generators one at a time (Procedure 1
// picks the minimum unexpanded entry, Procedure 4 relaxes every vertex that
// sees it). Here the same costs are reached as the fixpoint of
//     cost(v) = min over generators u that see v, with v inside u's shadow
//               cone, of cost(u) + |u - v|
// computed on the GPU in three steps:
//   1. k_vis_pairs: one bit per (generator u, obstacle vertex v) pair, set when
//      u sees v exactly and the line uv is tangent to the obstacle wedges of u
//      and of v (a vertex passes a path on only along a tangent: other edges
//      never carry a shortest path to a pixel); segment interiors reach v
//      through its perpendicular foot. A vertex whose shortest arrival is not
//      tangent has an empty shadow cone and is never a parent, so only its
//      own reported cost can exceed the true one. The local depth maps of
//      the obstacle vertices (k_vert_maps, once per scene) reject most hidden
//      pairs before the exact test.
//   2. k_edges_*: the bits become CSR in-lists (by v) with FP64 edge lengths
//      and out-lists (by u) for frontier marking.
//   3. k_sssp_solo: for sparse graphs, one CTA with the graph in shared
//      memory runs rounds over the vertices whose in-neighbours changed, each
//      pulling its in-neighbours' current state; k_sssp_cluster: for denser
//      ones, the same rounds on one thread-block cluster with the state
//      replicated in every CTA; k_sssp: otherwise, the rounds (synchronous)
//      on every SM with a cooperative launch. All stop at the fixpoint
//      (bounded round count -> status bit).
// On deep graphs the rounds start from a shortest-path tree of the obstacle
// vertices' geodesic table (k_warm_*, below), whose first three kernels run
// while the edge lists are built on a second stream.
// Costs are FP64 with explicitly rounded operations, so they match a plain
// FP64 Dijkstra over the same edges bit for bit.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>
#include <atomic>
#include <cuda_runtime.h>

#include "spm_device.cuh"
#include "spm_internal.h"

namespace spm {
// Programmatic dependent launch along the vertex phase's chain of small
// kernels: a kernel launched with programmatic stream serialization may be
// scheduled while its predecessor in the stream still runs. Each chain
// kernel first lets its own successor be scheduled (launch_dependents), then
// waits (griddepcontrol.wait) until its predecessor has completed and that
// grid's memory is visible, before it reads anything. Launched the ordinary
// way, both instructions do nothing.
__device__ __forceinline__ void chain_start() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
}  // namespace spm

namespace cg = cooperative_groups;

namespace spm {
namespace {

constexpr int kVisThreads = 256;
constexpr int kSsspThreads = 256;
#ifndef SPM_SOLO_THREADS
#define SPM_SOLO_THREADS 512
#endif
constexpr int kSoloThreads = SPM_SOLO_THREADS;  // threads of the single-CTA fixpoint
#ifndef SPM_SOLO_GRP
#define SPM_SOLO_GRP 8
#endif
constexpr int kSoloGrp = SPM_SOLO_GRP;  // lanes per dirty vertex in the single-CTA fixpoint (in-degrees are small)
#ifndef SPM_SOLO_MAX_DEG
#define SPM_SOLO_MAX_DEG 8
#endif
constexpr int kSoloSmem = 226 * 1024;  // within the 227 KB opt-in maximum, with the static part

// Static filter for one (u, v) pair: tangency at both ends, or for a
// segment interior u a perpendicular foot strictly inside the segment.
__device__ bool pair_filter(const DevScene &ds, int u, int v) {
    if (u == v) return false;
    const int ku = ds.gen_kind[u];
    const int2 vl = ds.gen_lat[v];
    if (ku == kSegI) {
        const int4 L = ds.seg_lat[ds.gen_aux[u]];
        const long long ux = L.z - L.x, uy = L.w - L.y;
        const long long num = (vl.x - L.x) * ux + (vl.y - L.y) * uy;
        return num > 0 && num < ux * ux + uy * uy;
    }
    const int2 ul = ds.gen_lat[u];
    if (ul.x == vl.x && ul.y == vl.y) return false;
    const int wx = vl.x - ul.x, wy = vl.y - ul.y;
    if (ku == kVert) {  // tangent at u: the line uv does not split u's wedge
        const int4 w = ds.gen_wedge[u];
        const int a = cross32(wx, wy, w.x, w.y), b = cross32(wx, wy, w.z, w.w);
        if ((a > 0 && b < 0) || (a < 0 && b > 0)) return false;
    }
    // tangent at v: an arrival pointing into v's wedge leaves v an empty
    // shadow cone, so v could never pass such a path on
    const int4 w = ds.gen_wedge[v];
    const int a = cross32(wx, wy, w.x, w.y), b = cross32(wx, wy, w.z, w.w);
    return !((a > 0 && b < 0) || (a < 0 && b > 0));
}

// Local depth maps (obstacles are fixed, so they are built once per scene).
// Directions around a vertex are cut into kLocBins bins of the pseudo-angle;
// map[b] bounds from above the squared distance at which every ray of bin b
// has crossed a front-facing edge of a nearby polygon (the vertex strictly
// on the edge's outer side), i.e. entered that polygon's interior. Along an
// edge's line the crossing distance is convex in the ray angle, so over a
// bin it peaks at a boundary ray; boundary directions are integer vectors
// (multiples of 1 / kLocQ per quadrant), so the products are exact in
// integers up to a few float roundings, covered by a 1e-5 relative margin.
// Only polygons of the bins within two bins of the vertex enter; leaving
// others out only raises the bounds.
constexpr int kLocQ = kLocBins / 4;
constexpr float kLocW = 4.0f / kLocBins;

__device__ __forceinline__ int2 loc_boundary_dir(int m) {
    const int mm = m & (kLocBins - 1), f = mm & (kLocQ - 1);
    switch (mm / kLocQ) {
        case 0: return make_int2(kLocQ - f, f);
        case 1: return make_int2(-f, kLocQ - f);
        case 2: return make_int2(-(kLocQ - f), -f);
        default: return make_int2(f, -(kLocQ - f));
    }
}

// One warp per obstacle vertex; the lanes over the bins an edge spans.
__global__ void __launch_bounds__(256) k_vert_maps(const __grid_constant__ DevScene ds, float *maps) {
    __shared__ float sm[8][kLocBins];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int vv = blockIdx.x * 8 + warp;
    if (vv >= ds.n_vert) return;  // whole warps
    float *map = sm[warp];
    for (int k = lane; k < kLocBins; k += 32) map[k] = INFINITY;
    __syncwarp();
    const int2 g = ds.gen_lat[ds.n_src + vv];
    const int cx = (g.x - ds.bin_x0) / ds.bin_size, cy = (g.y - ds.bin_y0) / ds.bin_size;
    for (int by = max(0, cy - 2); by <= min(ds.bin_ny - 1, cy + 2); ++by)
        for (int bx = max(0, cx - 2); bx <= min(ds.bin_nx - 1, cx + 2); ++bx) {
            const int bin = by * ds.bin_nx + bx;
            for (int it = ds.bin_start[bin]; it < ds.bin_start[bin + 1]; ++it) {
                const BinRec rec = ds.bin_recs[it];
                const int2 *V = ds.poly_v + rec.voff;
                for (int i = 0; i < rec.m; ++i) {
                    const int2 a = V[i], c = V[i + 1 == rec.m ? 0 : i + 1];
                    if (orient32(a.x, a.y, c.x, c.y, g.x, g.y) >= 0) continue;  // not front-facing
                    const int nx = -(c.y - a.y), ny = c.x - a.x;
                    const long long N = (long long)nx * (a.x - g.x) + (long long)ny * (a.y - g.y);
                    const float fN2 = (float)N * (float)N;
                    // the edge runs clockwise seen from g: counter-clockwise from c to a
                    const float lo = pang((float)(c.x - g.x), (float)(c.y - g.y));
                    const float hi = lo + fmodf(pang((float)(a.x - g.x), (float)(a.y - g.y)) - lo + 4.f, 4.f);
                    const int k0 = (int)ceilf((lo + kAngEps) / kLocW), k1 = (int)floorf((hi - kAngEps) / kLocW) - 1;
                    auto bdist2 = [&](int mb) {
                        const int2 u = loc_boundary_dir(mb);
                        const float fD = (float)(nx * u.x + ny * u.y);  // exact: |n| < 2^16, |u| <= kLocQ
                        return __fdividef(fN2 * (float)(u.x * u.x + u.y * u.y), fD * fD) * (1.f + 1e-5f);
                    };
                    for (int k = k0 + lane; k <= k1; k += 32) {
                        int *slot = (int *)&map[k & (kLocBins - 1)];
                        atomicMin(slot, __float_as_int(fmaxf(bdist2(k), bdist2(k + 1))));
                    }
                }
            }
        }
    __syncwarp();
    for (int k = lane; k < kLocBins; k += 32) maps[(size_t)vv * kLocBins + k] = map[k];
}

// Is lattice point q hidden from obstacle vertex v by v's local depth map?
__device__ __forceinline__ bool loc_hidden(const DevScene &ds, int v, int2 vl, int2 q) {
    const int rx = q.x - vl.x, ry = q.y - vl.y;
    const float r2 = (float)((long long)rx * rx + (long long)ry * ry);
    const float a = pang((float)rx, (float)ry);
    const int b0 = (int)floorf((a - kAngEps) / kLocW), b1 = (int)floorf((a + kAngEps) / kLocW);
    const float *map = ds.vert_maps + (size_t)(v - ds.n_src) * kLocBins;
    return r2 * (1.f - 1e-5f) >= fmaxf(__ldg(map + ((b0 + kLocBins) & (kLocBins - 1))),
                                       __ldg(map + (b1 & (kLocBins - 1))));
}

// Exact visibility of a pair that passed the filter. The predicate is
// symmetric in the two ends; a source's pairs are walked from the source,
// since the vertex end already passed its local depth map (what blocks such
// a pair lies farther from the vertex, often near the source).
__device__ bool pair_visible(const DevScene &ds, int u, int v) {
    const int2 vl = ds.gen_lat[v];
    if (ds.gen_kind[u] == kSegI) {
        const int s = ds.gen_aux[u];
        const int4 L = ds.seg_lat[s];
        const long long ux = L.z - L.x, uy = L.w - L.y;
        return visible_foot(ds, s, vl.x, vl.y, (vl.x - L.x) * ux + (vl.y - L.y) * uy, ux * ux + uy * uy, true);
    }
    const int2 ul = ds.gen_lat[u];
    return u < ds.n_src ? visible_points(ds, ul.x, ul.y, vl.x, vl.y) : visible_points(ds, vl.x, vl.y, ul.x, ul.y);
}

// Sets the bit of edge u -> v (row v) and, between two obstacle vertices,
// its mirror v -> u (row u). The matrix starts zeroed.
__device__ __forceinline__ void set_edge_bits(const DevScene &ds, int u, int v) {
    atomicOr(&ds.vis_bits[(size_t)(v - ds.n_src) * ds.vis_words + (u >> 5)], 1u << (u & 31));
    if (u >= ds.n_src) atomicOr(&ds.vis_bits[(size_t)(u - ds.n_src) * ds.vis_words + (v >> 5)], 1u << (v & 31));
}

// Visibility pairs of one or many scenes. A warp task is row vv (vertex
// index) of a scene's bit matrix and word w covering generators
// 32w..32w+31. A pair of obstacle vertices passes the filter and sees each
// other symmetrically (both tangency tests and the blocking predicate are
// symmetric in the two points), so only generators u < v are tested and an
// edge between two vertices also sets its mirror bit. Pairs that pass the
// filter queue up per warp in shared memory and are walked 32 at a time, so
// every lane walks (the filter passes a few lanes of each word).
constexpr int kPairQ = 64;
struct PairQ {
    int3 e[kVisThreads / 32][kPairQ];  // (scene, u, v)
};

// Warps take tasks `chunk` at a time, the first by their index, the rest
// from a work counter: the walks left after the filters are few and uneven,
// and a fixed share per warp leaves SMs idle behind a few long ones. A chunk
// is a run of consecutive words of one row, so the row vertex's data and
// local map stay in L1; the host sizes it so that every resident warp takes
// about two chunks.
template <class Scene, class Task>
__device__ __forceinline__ void vis_pairs_run(PairQ &q, long long tasks, int chunk, unsigned long long *work,
                                              Scene scene_of_task, Task task_of) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int qn = 0;  // warp-uniform queue length
    auto walk = [&](int n) {  // lanes < n walk the last n queued pairs
        if (lane < n) {
            const int3 pr = q.e[warp][qn - n + lane];
            const DevScene &ds = *scene_of_task(pr.x);
            const bool vis = pair_visible(ds, pr.y, pr.z);
            if (vis) set_edge_bits(ds, pr.y, pr.z);
            SPM_CNT(13, 1);
            SPM_CNT(14, vis ? 1 : 0);
        }
        qn -= n;
        __syncwarp();
    };
    // Each warp's first chunk is its own by its index (thousands of warps
    // starting on one counter would queue on its atomics); the rest come
    // from the counter, after those.
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5), gw = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    const long long handed = nw * chunk;
    long long t = 0, t_end = 0;
    bool first = true;
    for (;;) {
        if (t == t_end) {
            if (first) {
                first = false;
                t = gw * chunk;
            } else {
                if (handed >= tasks) break;  // every task was handed out by index
                unsigned long long c = 0;
                if (lane == 0) c = atomicAdd(work, (unsigned long long)chunk);
                t = handed + (long long)__shfl_sync(0xffffffffu, c, 0);
            }
            if (t >= tasks) break;
            t_end = min(t + chunk, tasks);
        }
        const long long tt = t++;
        int sc;
        long long lt;
        task_of(tt, sc, lt);
        const DevScene &ds = *scene_of_task(sc);
        const int vv = (int)(lt / ds.pair_words), w = (int)(lt % ds.pair_words);
        const int u = w * 32 + lane, v = ds.n_src + vv;
        if (w * 32 >= v) continue;  // the whole word lies at or above the diagonal (warp-uniform)
        bool c = u < v && u >= ds.pair_u0 && u < ds.pair_u1 && pair_filter(ds, u, v);
        if (c && ds.vert_maps && ds.gen_kind[u] != kSegI) {  // hidden by an obstacle near either end
            const int2 ul = ds.gen_lat[u], vl = ds.gen_lat[v];
            c = !loc_hidden(ds, v, vl, ul) && !(u >= ds.n_src && loc_hidden(ds, u, ul, vl));
        }
        const unsigned bal = __ballot_sync(0xffffffffu, c);
        if (c) q.e[warp][qn + __popc(bal & ((1u << lane) - 1u))] = make_int3(sc, u, v);
        qn += __popc(bal);
        __syncwarp();
        if (qn >= 32) walk(32);
    }
    if (qn > 0) walk(qn);
}

__global__ void __launch_bounds__(kVisThreads) k_vis_pairs(const __grid_constant__ DevScene ds, int chunk) {
    __shared__ PairQ q;
    chain_start();
    vis_pairs_run(
        q, (long long)ds.n_vert * ds.pair_words, chunk, reinterpret_cast<unsigned long long *>(ds.stats + 2),
        [&](int) { return &ds; },
        [&](long long t, int &sc, long long &lt) {
            sc = 0;
            lt = t;
        });
}

// In-degree per vertex row and out-degree per generator: one warp per row,
// lanes over the row's words.
// With the static lists only the source columns are scanned (their out-
// degrees counted here; the obstacle vertices' come from st_out_init).
__device__ __forceinline__ uint32_t src_word_mask(const DevScene &ds, int w) {
    const int lo = ds.n_src - 32 * w;  // source columns in word w
    return lo >= 32 ? 0xffffffffu : lo <= 0 ? 0u : (1u << lo) - 1u;
}
__device__ __forceinline__ void edges_count_row(const DevScene &ds, int vv, int lane) {
    const uint32_t *row = ds.vis_bits + (size_t)vv * ds.vis_words;
    const bool st = ds.st_start != nullptr;
    const int nw = st ? (ds.n_src + 31) / 32 : ds.vis_words;
    int cnt = 0;
    for (int w = lane; w < nw; w += 32) {
        uint32_t b = row[w];
        if (st) b &= src_word_mask(ds, w);
        cnt += __popc(b);
        while (b) {
            const int bit = __ffs(b) - 1;
            b &= b - 1;
            atomicAdd(&ds.out_start[w * 32 + bit + 1], 1);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) ds.in_start[vv + 1] = cnt + (st ? ds.st_start[vv + 1] - ds.st_start[vv] : 0);
}

__global__ void k_edges_count(const __grid_constant__ DevScene ds) {
    chain_start();
    const int lane = threadIdx.x & 31, nw = gridDim.x * (blockDim.x >> 5);
    for (int vv = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); vv < ds.n_vert; vv += nw)
        edges_count_row(ds, vv, lane);
}

// Exclusive scans of in_start (n_vert + 1) and out_start (n_gen + 1), one CTA.
__device__ __forceinline__ void edges_scan_block(const DevScene &ds, long long *part) {
    for (int which = 0; which < 2; ++which) {
        int32_t *a = which == 0 ? ds.in_start : ds.out_start;
        const int n = which == 0 ? ds.n_vert : ds.n_gen;  // entries 1..n hold counts
        const int per = (n + blockDim.x - 1) / blockDim.x;
        const int lo = 1 + threadIdx.x * per, hi = min(n + 1, lo + per);
        long long s = 0;
        for (int i = lo; i < hi; ++i) s += a[i];
        long long run = cta_exclusive_scan(s, part);
        for (int i = lo; i < hi; ++i) {
            run += a[i];
            a[i] = (int32_t)min(run, (long long)INT32_MAX);
        }
        if (threadIdx.x == 0) a[0] = 0;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        long long E = ds.in_start[ds.n_vert];
        ds.stats[1] = (int32_t)E;
        if (E > ds.edge_cap) atomicOr(ds.status, kStEdgeOverflow);
    }
}

__global__ void __launch_bounds__(1024) k_edges_scan(const __grid_constant__ DevScene ds) {
    __shared__ long long part[32];
    chain_start();
    edges_scan_block(ds, part);
}

__device__ __forceinline__ double edge_len(const DevScene &ds, int u, int v) {
    const float2 vp = ds.gen_pos[v];
    if (ds.gen_kind[u] == kSegI) {
        const float4 F = ds.seg_pos[ds.gen_aux[u]];
        double ux = __dsub_rn((double)F.z, (double)F.x), uy = __dsub_rn((double)F.w, (double)F.y);
        double c = __dsub_rn(__dmul_rn(ux, __dsub_rn((double)vp.y, (double)F.y)),
                             __dmul_rn(uy, __dsub_rn((double)vp.x, (double)F.x)));
        return __ddiv_rn(fabs(c), __dsqrt_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy))));
    }
    const float2 up = ds.gen_pos[u];
    double dx = __dsub_rn((double)vp.x, (double)up.x), dy = __dsub_rn((double)vp.y, (double)up.y);
    return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

// In-list of row vv in generator order (the same order as a serial scan of
// the row): one warp, lanes over words, a warp prefix places each word.
__device__ __forceinline__ void edges_fill_row(const DevScene &ds, int vv, int lane) {
    const uint32_t *row = ds.vis_bits + (size_t)vv * ds.vis_words;
    int e0 = ds.in_start[vv];
    const int v = ds.n_src + vv;
    const bool st = ds.st_start != nullptr;
    const int nw = st ? (ds.n_src + 31) / 32 : ds.vis_words;
    for (int w0 = 0; w0 < nw; w0 += 32) {
        const int w = w0 + lane;
        uint32_t b = w < nw ? row[w] : 0u;
        if (st) b &= src_word_mask(ds, w);
        const int c = __popc(b);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        int e = e0 + inc - c;
        while (b) {
            const int u = w * 32 + __ffs(b) - 1;
            b &= b - 1;
            ds.in_src[e] = u;
            ds.in_len[e] = edge_len(ds, u, v);
            ++e;
            const int slot = atomicAdd(&ds.out_fill[u], 1);
            ds.out_dst[ds.out_start[u] + slot] = v;
        }
        e0 += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (st) {  // then the row's obstacle-vertex edges, as kept
        const int s0 = ds.st_start[vv], m = ds.st_start[vv + 1] - s0;
        for (int j = lane; j < m; j += 32) {
            ds.in_src[e0 + j] = ds.st_src[s0 + j];
            ds.in_len[e0 + j] = ds.st_len[s0 + j];
        }
    }
}

// An obstacle vertex's out-list, as kept, at its place in this compute's CSR.
__device__ __forceinline__ void edges_out_copy(const DevScene &ds, int uu, int lane) {
    const int b = ds.out_start[ds.n_src + uu], s0 = ds.st_out_start[uu], m = ds.st_out_start[uu + 1] - s0;
    for (int j = lane; j < m; j += 32) ds.out_dst[b + j] = ds.st_out_dst[s0 + j];
}

__global__ void k_edges_fill(const __grid_constant__ DevScene ds) {
    chain_start();
    if (ds.in_start[ds.n_vert] > ds.edge_cap) return;
    const int lane = threadIdx.x & 31, nw = gridDim.x * (blockDim.x >> 5);
    for (int vv = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); vv < ds.n_vert; vv += nw)
        edges_fill_row(ds, vv, lane);
    if (ds.st_start)
        for (int uu = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); uu < ds.n_vert; uu += nw)
            edges_out_copy(ds, uu, lane);
}

// FP64 lengths of the kept in-lists: the same function as a compute's.
__global__ void k_static_lengths(const __grid_constant__ DevScene ds, double *len) {
    const int lane = threadIdx.x & 31, nw = gridDim.x * (blockDim.x >> 5);
    for (int vv = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); vv < ds.n_vert; vv += nw)
        for (int e = ds.st_start[vv] + lane; e < ds.st_start[vv + 1]; e += 32)
            len[e] = edge_len(ds, ds.st_src[e], ds.n_src + vv);
}

// The finalised table entry of generator g (the pixel pass reads FP32 costs).
__device__ __forceinline__ void finalize_gen(const DevScene &ds, int g, double c, int p) {
    ds.gen_cost[g] = c;
    ds.gen_par[g] = p;
    ds.gen_costf[g] = (float)c;
}

// Jacobi rounds of the fixpoint on the whole GPU (cooperative launch, two
// grid barriers per round). cost[0]/par[0] and the cone cache hold the
// committed state; a round
//   pull:   one warp per dirty vertex v reduces its in-list to the
//           lexicographic minimum of (cost(u) + |u - v|, u) over valid u
//           (u a source, or v inside u's committed shadow cone) and records
//           v when that differs from its committed state;
//   commit: the changed vertices become committed (cost, parent, cone) and
//           mark their out-neighbours dirty for the next round.
// Lists and counters alternate by round parity, so a counter is zeroed only
// in a phase where nobody reads it. Stops when no vertex changes, or at the
// round cap (status bit). Deterministic: each pull is a min over a set.
__device__ __forceinline__ void commit_vertex(const DevScene &ds, int v) {
    ds.cost[0][v] = __ldcg(&ds.cost[1][v]);
    const int p = __ldcg(&ds.par[1][v]);
    ds.par[0][v] = p;
    int4 c = make_int4(0, 0, 0, 0);
    int ct = kConeEmpty;  // unreachable again: no arrival direction
    if (p >= 0) {
        int dx, dy;
        arrival_dir(ds, p, ds.gen_lat[v], dx, dy);
        ct = make_cone(ds.gen_wedge[v], dx, dy, c);
    }
    ds.gen_cone[v] = c;
    ds.gen_ctype[v] = ct;
}

// One warp marks the out-neighbours of u dirty, appending each newly dirty
// vertex once to the dirty list (warp-aggregated counter update).
__device__ __forceinline__ void mark_out_warp(const DevScene &ds, int u, int lane, int32_t *dl,
                                              int32_t *dcount) {
    const int e0 = ds.out_start[u], e1 = ds.out_start[u + 1];
    for (int eb = e0; eb < e1; eb += 32) {
        const int e = eb + lane;
        bool fresh = false;
        int v = 0;
        if (e < e1) {
            v = ds.out_dst[e];
            const uint32_t bit = 1u << (v & 31);
            fresh = !(atomicOr(&ds.dirty[v >> 5], bit) & bit);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, fresh);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(dcount, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (fresh) dl[base + __popc(bal & ((1u << lane) - 1u))] = v;
    }
}

// Shared-memory bytes the single-CTA fixpoint needs (0 if it cannot run).
// Shared memory of the single-CTA fixpoint, 0 when the graph does not fit or
// is not sparse. with_len: the FP64 edge lengths fit as well.
__host__ __device__ __forceinline__ int solo_bytes_for(long long n, int nv, long long E, long long edge_cap,
                                                       int solo_smem, bool &with_len) {
    with_len = false;
    // sparse graphs only (deep, few vertices per round); dense ones need more SMs
    if (n >= 32768 || E > edge_cap || E > SPM_SOLO_MAX_DEG * n) return 0;
    // cost 8, parent 2, lattice 4, wedge 8 per generator; CSR in / out with
    // 16-bit ids; two dirty bitmaps and lists; 16-byte alignment slack
    const long long b = n * (8 + 2 + 4 + 8) + 4 * (nv + 1) + 2 * E + 4 * (n + 1) + 2 * E +
                        2 * 4 * ((n + 31) / 32) + 2 * 2 * n + 16 * 16;
    if (b > solo_smem) return 0;
    with_len = b + 8 * E <= solo_smem;
    return (int)(with_len ? b + 8 * E : b);
}
__device__ __forceinline__ int solo_bytes(const DevScene &ds, bool &with_len) {
    return solo_bytes_for(ds.n_gen, ds.n_vert, ds.in_start[ds.n_vert], ds.edge_cap, ds.solo_smem, with_len);
}

__global__ void __launch_bounds__(256) k_sssp(const __grid_constant__ DevScene ds, int max_rounds) {
    bool solo_len;
    if (solo_bytes(ds, solo_len) > 0) return;  // the single-CTA kernel handles this graph
    if (ds.counters[4]) return;                // the cluster kernel did
    cg::grid_group grid = cg::this_grid();
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsize = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, gwarp = gtid >> 5, nwarps = gsize >> 5;
    const int n = ds.n_gen;
    int32_t *cnt = ds.counters;  // [0,1] frontier counts, [2,3] dirty counts
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    const bool overflow = ds.in_start[ds.n_vert] > ds.edge_cap;
    for (int g = gtid; g < n; g += gsize) {
        const bool src = g < ds.n_src;
        ds.cost[0][g] = src ? 0.0 : inf;
        ds.par[0][g] = src ? g : -1;
        ds.gen_ctype[g] = src ? kConeNone : kConeEmpty;
        ds.gen_cone[g] = make_int4(0, 0, 0, 0);
    }
    for (int w = gtid; w < (n + 31) / 32; w += gsize) ds.dirty[w] = 0u;
    if (gtid < 4) cnt[gtid] = 0;
    grid.sync();
    if (!overflow)
        for (int u = gwarp; u < ds.n_src; u += nwarps) mark_out_warp(ds, u, lane, ds.dirtyl[0], &cnt[2]);
    grid.sync();
    int round = 0;
    for (;; ++round) {
        const int par_r = round & 1, par_n = par_r ^ 1;
        // pull
        if (gtid == 0) {
            cnt[par_n] = 0;
            cnt[2 + par_n] = 0;
        }
        // data written by other CTAs since the last grid barrier is read
        // through L2 (__ldcg): L1 is not coherent across SMs
        const int nd = __ldcg(&cnt[2 + par_r]);
        const int32_t *dl = ds.dirtyl[par_r];
        for (int i = gwarp; i < nd; i += nwarps) {
            const int v = __ldcg(&dl[i]);
            const int vv = v - ds.n_src;
            if (lane == 0) atomicAnd(&ds.dirty[v >> 5], ~(1u << (v & 31)));
            const int2 vl = ds.gen_lat[v];
            long long best = 0x7ff0000000000000ll;  // +inf bits
            int bpar = -1;
            for (int e = ds.in_start[vv] + lane; e < ds.in_start[vv + 1]; e += 32) {
                const int u = ds.in_src[e];
                const double cu = __ldcg(&ds.cost[0][u]);
                if (__double_as_longlong(cu) >= 0x7ff0000000000000ll) continue;  // unreached
                const int ct = __ldcg(&ds.gen_ctype[u]);
                if (ct != kConeNone) {
                    const int2 ul = ds.gen_lat[u];
                    if (!in_cone(ct, __ldcg(&ds.gen_cone[u]), vl.x - ul.x, vl.y - ul.y)) continue;
                }
                // costs are non-negative, so their bit patterns order like
                // their values: compare as integers, keep FP64 for the add
                const long long cand = __double_as_longlong(__dadd_rn(cu, ds.in_len[e]));
                if (cand < best || (cand == best && u < bpar)) {
                    best = cand;
                    bpar = u;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int op = __shfl_xor_sync(0xffffffffu, bpar, o);
                if (ob < best || (ob == best && (unsigned)op < (unsigned)bpar)) {
                    best = ob;
                    bpar = op;
                }
            }
            if (lane == 0 && (best != __double_as_longlong(__ldcg(&ds.cost[0][v])) || bpar != __ldcg(&ds.par[0][v]))) {
                ds.cost[1][v] = __longlong_as_double(best);
                ds.par[1][v] = bpar;
                ds.frontier[par_r][atomicAdd(&cnt[par_r], 1)] = v;
            }
        }
        grid.sync();
        const int nc = __ldcg(&cnt[par_r]);
        if (nc == 0) break;
        if (round + 1 >= max_rounds) {
            if (gtid == 0) atomicOr(ds.status, kStNotConverged);
            break;
        }
        // commit the changed vertices and mark their out-neighbours
        const int32_t *fr = ds.frontier[par_r];
        for (int i = gtid; i < nc; i += gsize) commit_vertex(ds, __ldcg(&fr[i]));
        for (int i = gwarp; i < nc; i += nwarps) mark_out_warp(ds, __ldcg(&fr[i]), lane, ds.dirtyl[par_n], &cnt[2 + par_n]);
        grid.sync();
    }
    if (gtid == 0) ds.stats[0] = round + 1;
}

// The same fixpoint in one CTA with the graph and the state in shared
// memory, for graphs that fit (16-bit generator ids and lattice coordinates;
// wedge directions are lattice differences and fit in 16 bits as well). One
// barrier per round. A dirty vertex pulls its in-neighbours' current state --
// including values written earlier in the same round, so a change can travel
// several edges in one round -- and, when its own value changes, writes it and
// marks its out-neighbours in the next round's dirty bitmap and list. A
// neighbour's shadow cone is derived from its current parent when it is
// pulled. A pull may see a neighbour half-way through an update in the same
// round; that neighbour's change marks the puller dirty again, so the last
// round reads only settled values and the loop stops at the fixpoint of the
// vertex equations. With positive link lengths that fixpoint is unique
// (costs and then parents are fixed in order of increasing cost), so the
// result is the one k_sssp's synchronous rounds reach. The FP64 link
// lengths are staged in shared memory when they fit, else read from global.
//
// A round is one dependent chain per dirty vertex, so it is laid out for
// latency: everything a group needs about its vertex is loaded in one level,
// the kinds and lattice endpoints of the first sources sit in shared memory
// (a segment-interior parent needs no global load), the out-neighbours are
// marked with one counter atomic per warp, and the finished round's dirty
// bitmap is cleared in bulk.
constexpr int kSoloSrc = 32;  // sources whose kind and segment endpoints are staged

#ifdef SPM_COUNT
// clock read ordered after the value x has been computed (instrumentation)
template <class T>
__device__ __forceinline__ long long clock_after(T x) {
    asm volatile("" ::"l"((long long)x) : "memory");
    return clock64();
}
#endif

__device__ __forceinline__ void arrival_from(const DevScene &ds, const signed char *src_kind, const int4 *src_seg,
                                             const short2 *lat, int p, short2 vl, int &dx, int &dy) {
    if (p >= ds.n_src || (p < kSoloSrc ? src_kind[p] : ds.gen_kind[p]) != kSegI) {
        dx = vl.x - lat[p].x;
        dy = vl.y - lat[p].y;
        return;
    }
    // segment interior: perpendicular to the segment, toward v
    const int4 L = p < kSoloSrc ? src_seg[p] : ds.seg_lat[ds.gen_aux[p]];
    const int ux = L.z - L.x, uy = L.w - L.y;
    const int side = cross32(ux, uy, vl.x - L.x, vl.y - L.y);
    dx = side > 0 ? -uy : uy;
    dy = side > 0 ? ux : -ux;
}

// Copies n 4-byte words from global to shared memory (both 16-byte
// aligned) by asynchronous 16-byte copies, the tail word by word; the caller
// waits (cp.async.wait_all) before its barrier.
__device__ __forceinline__ void async_copy_words(void *dst, const void *src, long long n, int tid, int nthr) {
    const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(dst);
    const char *s0 = (const char *)src;
    const long long n4 = n / 4;
    for (long long i = tid; i < n4; i += nthr)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d0 + 16 * (uint32_t)i), "l"(s0 + 16 * i) : "memory");
    for (long long i = 4 * n4 + tid; i < n; i += nthr)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d0 + 4 * (uint32_t)i), "l"(s0 + 4 * i) : "memory");
}

// n int32 generator ids (global, 16-byte aligned) into 16-bit ids in shared
// memory (8-byte aligned), four per 16-byte load.
__device__ __forceinline__ void narrow_ids(unsigned short *dst, const int32_t *src, int n, int tid, int nthr) {
    const int n4 = n / 4;
#pragma unroll 4
    for (int i = tid; i < n4; i += nthr) {
        const int4 a = __ldg(reinterpret_cast<const int4 *>(src) + i);
        reinterpret_cast<ushort4 *>(dst)[i] =
            make_ushort4((unsigned short)a.x, (unsigned short)a.y, (unsigned short)a.z, (unsigned short)a.w);
    }
    for (int i = 4 * n4 + tid; i < n; i += nthr) dst[i] = (unsigned short)src[i];
}

__global__ void __launch_bounds__(kSoloThreads) k_sssp_solo(const __grid_constant__ DevScene ds, int max_rounds) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    chain_start();
#ifdef SPM_COUNT
    const long long t_start = clock64();
#endif
    bool with_len;
    if (solo_bytes(ds, with_len) == 0) return;
    const int n = ds.n_gen, nv = ds.n_vert, E = ds.in_start[nv];
    unsigned char *p = sm_raw;
    auto take = [&](size_t sz) {
        unsigned char *q = p;
        p += (sz + 15) & ~(size_t)15;
        return q;
    };
    double *cost = (double *)take(8 * (size_t)n);
    short4 *wedge = (short4 *)take(8 * (size_t)n);
    short *par = (short *)take(2 * (size_t)n);
    short2 *lat = (short2 *)take(4 * (size_t)n);
    int *in_start = (int *)take(4 * (size_t)(nv + 1));
    unsigned short *in_src = (unsigned short *)take(2 * (size_t)E);
    int *out_start = (int *)take(4 * (size_t)(n + 1));
    unsigned short *out_dst = (unsigned short *)take(2 * (size_t)E);
    const int dw = (n + 31) / 32;
    unsigned *dirty = (unsigned *)take(4 * 2 * (size_t)dw);         // round parity p at p * dw
    unsigned short *dl = (unsigned short *)take(2 * 2 * (size_t)n);  // round parity p at p * n
    double *slen = with_len ? (double *)take(8 * (size_t)E) : nullptr;
    __shared__ int cnt[3];  // dirty-list counts, by round modulo 3
    __shared__ signed char src_kind[kSoloSrc];  // kinds of the first sources (ids >= n_src are vertices)
    __shared__ int4 src_seg[kSoloSrc];          // their segment's lattice endpoints (segment sources)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kSoloThreads / 32;
    // work unit: a group of kSoloGrp lanes per dirty vertex
    constexpr int kGpw = 32 / kSoloGrp;  // groups per warp
    const int grp = lane / kSoloGrp, gl = lane % kSoloGrp, ngroups = nwarps * kGpw;
    const unsigned kFull = 0xffffffffu;
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    // arrays copied as they are go by asynchronous copies (many in flight,
    // no registers); the 16-bit ids are narrowed from 16-byte loads
    async_copy_words(in_start, ds.in_start, nv + 1, tid, kSoloThreads);
    async_copy_words(out_start, ds.out_start, n + 1, tid, kSoloThreads);
    if (with_len) async_copy_words(slen, ds.in_len, 2 * E, tid, kSoloThreads);
    narrow_ids(in_src, ds.in_src, E, tid, kSoloThreads);
    narrow_ids(out_dst, ds.out_dst, E, tid, kSoloThreads);
#pragma unroll 4
    for (int g = tid; g < n; g += kSoloThreads) {
        const bool src = g < ds.n_src;
        cost[g] = ds.warm ? ds.warm_cost[g] : src ? 0.0 : inf;  // warm: the tree's state
        par[g] = (short)(ds.warm ? ds.warm_par[g] : src ? g : -1);
        const int2 l = ds.gen_lat[g];
        lat[g] = make_short2((short)l.x, (short)l.y);
        const int4 w = ds.gen_wedge[g];
        wedge[g] = make_short4((short)w.x, (short)w.y, (short)w.z, (short)w.w);
    }
    for (int w = tid; w < 2 * dw; w += kSoloThreads) dirty[w] = 0u;
    for (int g = tid; g < min(ds.n_src, kSoloSrc); g += kSoloThreads) {
        const int k = ds.gen_kind[g];
        src_kind[g] = (signed char)k;
        src_seg[g] = k == kSegI ? ds.seg_lat[ds.gen_aux[g]] : make_int4(0, 0, 0, 0);
    }
    if (tid < 3) cnt[tid] = 0;
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (ds.warm) {  // round 0 pulls the vertices whose equation the tree's state breaks
        const int m = min(ds.counters[6], nv);
        for (int i = tid; i < m; i += kSoloThreads) {
            const int v = ds.dirtyl[0][i];
            dl[i] = (unsigned short)v;
            atomicOr(&dirty[v >> 5], 1u << (v & 31));
        }
        if (tid == 0) cnt[0] = m;
    } else {  // the sources mark their out-neighbours for round 0
        for (int u = warp * kGpw + grp; u < ds.n_src; u += ngroups)
            for (int e = out_start[u] + gl; e < out_start[u + 1]; e += kSoloGrp) {
                const int v = out_dst[e];
                const unsigned bit = 1u << (v & 31);
                if (!(atomicOr(&dirty[v >> 5], bit) & bit)) dl[atomicAdd(&cnt[0], 1)] = (unsigned short)v;
            }
    }
    __syncthreads();
#ifdef SPM_COUNT
    if (tid == 0) SPM_CNT(15, clock64() - t_start);  // the graph's loads and the first marks
#endif
    int round = 0;
    for (;; ++round) {
        const int cur = round & 1, nxt = cur ^ 1;
        const int nd = cnt[round % 3];
        if (nd == 0) break;
        if (round >= max_rounds) {
            if (tid == 0) atomicOr(ds.status, kStNotConverged);
            break;
        }
        if (tid == 0) cnt[(round + 2) % 3] = 0;  // read last round, marked into next round
        int *next_cnt = &cnt[(round + 1) % 3];
#ifdef SPM_COUNT
        const long long t_round = clock64();
        if (tid == 0) {
            SPM_CNT(0, nd);
            SPM_CNT_MAX(1, nd);
        }
        long long lap[6] = {0, 0, 0, 0, 0, 0};
#endif
        for (int i0 = warp * kGpw; i0 < nd; i0 += ngroups) {  // warp-uniform trip count
            const int i = i0 + grp;
            const bool act = i < nd;
            const int v_list = dl[cur * n + min(i, n - 1)];  // loaded before nd is known
            const int v = act ? v_list : ds.n_src;
            const int vv = v - ds.n_src;
            // one level of loads: the vertex's lists, position and state
            const int e0 = in_start[vv] + gl, e1 = act ? in_start[vv + 1] : 0;
            const int o0 = out_start[v] + gl, o1 = act ? out_start[v + 1] : 0;
            const short2 vl = lat[v];
            const long long cv = __double_as_longlong(cost[v]);
            const int pv = par[v];
            long long best = 0x7ff0000000000000ll;  // +inf bits
            int bpar = -1;
#ifdef SPM_COUNT
            lap[0] = clock_after((long long)e1 + o1 + vl.x + cv + pv);  // the vertex's own loads
#endif
            const int o_first = out_dst[min(o0, E > 0 ? E - 1 : 0)];  // first out-neighbour, loaded early
            // The in-list runs in increasing generator order, so within a lane
            // the first of equal keys has the smaller id: a strict compare
            // keeps it. The pull is branch-free: divergent branches here cost
            // more than computing every test.
            for (int e = e0; e < e1; e += kSoloGrp) {
                const double len = with_len ? slen[e] : __ldg(ds.in_len + e);
                const int u = in_src[e];
                const double cu = cost[u];
                const int pu = par[u];
                const short2 ul = lat[u];
                const short4 w = wedge[u];
                // u's arrival direction: from its parent, or perpendicular to a
                // segment source whose interior is the parent
                const int pc = pu < 0 ? 0 : pu, ps = pc < kSoloSrc ? pc : 0;
                const short2 pl = lat[pc];
                const int4 L = src_seg[ps];
                int dx = ul.x - pl.x, dy = ul.y - pl.y;
                if (pu < ds.n_src && pu >= kSoloSrc) {  // beyond the staged sources (rare)
                    arrival_from(ds, src_kind, src_seg, lat, pu, ul, dx, dy);
                } else if (pu >= 0 && pu < ds.n_src && src_kind[ps] == kSegI) {
                    const int sx = L.z - L.x, sy = L.w - L.y;
                    const int side = cross32(sx, sy, ul.x - L.x, ul.y - L.y);
                    dx = side > 0 ? -sy : sy;
                    dy = side > 0 ? sx : -sx;
                }
                // an obstacle vertex passes paths on only inside its shadow cone
                const bool valid = (__double_as_longlong(cu) < 0x7ff0000000000000ll) &
                                   ((u < ds.n_src) | ((pu >= 0) & in_shadow_cone(dx, dy, w, vl.x - ul.x, vl.y - ul.y)));
                // costs are non-negative, so their bit patterns order like
                // their values: compare as integers, keep FP64 for the add
                const long long cand = __double_as_longlong(__dadd_rn(cu, len));
                const bool better = valid & (cand < best);
                best = better ? cand : best;
                bpar = better ? u : bpar;
            }
#ifdef SPM_COUNT
            lap[1] = clock_after(best + bpar);  // the pull
#endif
#pragma unroll
            for (int o = kSoloGrp / 2; o > 0; o >>= 1) {  // within the group
                const long long ob = __shfl_xor_sync(kFull, best, o);
                const int op = __shfl_xor_sync(kFull, bpar, o);
                if (ob < best || (ob == best && (unsigned)op < (unsigned)bpar)) {
                    best = ob;
                    bpar = op;
                }
            }
            // every lane of the group holds the group's result and the old state
            const bool changed = act && (best != cv || bpar != pv);
#ifdef SPM_COUNT
            lap[2] = clock_after(best + bpar);  // the reduction
#endif
            if (changed && gl == 0) {
                cost[v] = __longlong_as_double(best);  // only this group writes v in this round
                par[v] = (short)bpar;
            }
            // mark the out-neighbours (each newly dirty one once in the next list)
            if (changed)
                for (int e = o0; e < o1; e += kSoloGrp) {
                    const int w = e == o0 ? o_first : out_dst[e];
                    const unsigned bit = 1u << (w & 31);
                    if (!(atomicOr(&dirty[nxt * dw + (w >> 5)], bit) & bit)) dl[nxt * n + atomicAdd(next_cnt, 1)] = (unsigned short)w;
                }
#ifdef SPM_COUNT
            lap[3] = clock_after(changed);  // the marks
#endif
        }
        // this round's bitmap is free again (marks went to the other one); the
        // last threads clear it, whose warps rarely hold a dirty vertex
        for (int w = kSoloThreads - 1 - tid; w < dw; w += kSoloThreads) dirty[cur * dw + w] = 0u;
#ifdef SPM_COUNT
        if (lane == 0) SPM_CNT_MAX(6, (unsigned long long)(clock64() - t_round));  // slowest warp, any round
        if (tid == 0) {
            SPM_CNT(7, (unsigned long long)(clock64() - t_round));  // warp 0 (always has work)
            SPM_CNT(8, (unsigned long long)(lap[0] - t_round));     // list entry and the vertex's loads
            SPM_CNT(9, (unsigned long long)(lap[1] - lap[0]));      // pull over the in-edges
            SPM_CNT(10, (unsigned long long)(lap[2] - lap[1]));     // group reduction
            SPM_CNT(11, (unsigned long long)(lap[3] - lap[2]));     // commit and marks
        }
#endif
        __syncthreads();
#ifdef SPM_COUNT
        if (tid == 0) SPM_CNT(5, (unsigned long long)(clock64() - t_round));  // whole round, barrier included
#endif
    }
    // the settled state, with each vertex's shadow cone from its parent
    for (int g = tid; g < n; g += kSoloThreads) {
        const int pg = par[g];
        int4 c = make_int4(0, 0, 0, 0);
        int ct = kConeNone;
        if (g >= ds.n_src) {
            ct = kConeEmpty;  // unreached: no arrival direction
            if (pg >= 0) {
                int dx, dy;
                arrival_from(ds, src_kind, src_seg, lat, pg, lat[g], dx, dy);
                const short4 w = wedge[g];
                ct = make_cone(make_int4(w.x, w.y, w.z, w.w), dx, dy, c);
            }
        }
        ds.cost[0][g] = cost[g];
        ds.par[0][g] = pg;
        ds.gen_cone[g] = c;
        ds.gen_ctype[g] = ct;
        finalize_gen(ds, g, cost[g], pg);
    }
    if (tid == 0) ds.stats[0] = round;
}

// The fixpoint of graphs too dense for one CTA: one cluster of C CTAs (16
// where the GPU holds such a cluster, else 8; the batched form's are 8), one
// per SM, with the generators' state (cost, parent, lattice position, wedge,
// arrival direction) replicated in every CTA's shared memory and the
// obstacle vertices dealt round-robin to the CTAs, each holding the in-lists
// of its own. A round works as in the single-CTA kernel (a dirty vertex pulls
// the current state of its in-neighbours), but a changed vertex writes its
// value into every CTA's copy and sets its bit in every CTA's bitmap of
// changed generators, through distributed shared memory; after the round's
// cluster barrier each CTA finds its own dirty vertices by scanning their
// in-lists against that bitmap. One cluster barrier per round replaces the
// grid barriers of the many-CTA kernel. The argument of the single-CTA
// kernel carries over: a pull may read a neighbour mid-update, whose change
// marks the puller again, so the loop stops at the fixpoint of the vertex
// equations, which is unique.
constexpr int kClCtas = 8;          // CTAs of the batched form's clusters (the portable size)
constexpr int kClCtasWide = 16;     // CTAs of a single scene's cluster where the GPU holds one (non-portable)
constexpr int kClThreads = 1024;
constexpr int kClGrp = 16;          // lanes per dirty vertex (dense in-lists); at least the cluster's CTAs
constexpr int kClSmem = 200 * 1024; // dynamic shared memory per CTA

// The cluster fixpoint's layout: the replicated state and the dirty lists at
// offsets every CTA shares, then the CTA's own in-lists (with their FP64
// lengths when they fit; else the lengths are read from global memory).
struct ClLayout {
    size_t cost, wedge, par, lat, ldir, chg, dl, lin_start, gstart, lin_src, lin_len, end;
};
__host__ __device__ __forceinline__ ClLayout cl_layout(int n, int nv, long long e_own, bool with_len, int C) {
    auto up = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const int nmax = (nv + C - 1) / C;
    ClLayout L;
    L.cost = 0;
    L.wedge = L.cost + up(8 * (size_t)n);
    L.par = L.wedge + up(8 * (size_t)n);
    L.lat = L.par + up(2 * (size_t)n);
    L.ldir = L.lat + up(4 * (size_t)n);
    L.chg = L.ldir + up(8 * (size_t)n);
    L.dl = L.chg + up(4 * 2 * (((size_t)n + 31) / 32));
    L.lin_start = L.dl + up(2 * 2 * (size_t)nmax);
    L.gstart = L.lin_start + up(4 * ((size_t)nmax + 1));
    L.lin_src = L.gstart + up(4 * (size_t)nmax);
    L.lin_len = L.lin_src + up(2 * (size_t)e_own);
    L.end = L.lin_len + (with_len ? up(8 * (size_t)e_own) : 0);
    return L;
}

// Per-CTA static shared state of the cluster fixpoint.
struct ClShared {
    int cnt[3];                  // dirty-list counts, by round modulo 3
    long long own_e[kClCtasWide]; // in-edges of each CTA's vertices
    int next;                    // the batched form's next scene (CTA 0)
    long long wsum[32];
    signed char src_kind[kSoloSrc];
    int4 src_seg[kSoloSrc];
};

// One scene's fixpoint on the calling cluster of C CTAs (every thread of it
// calls). Returns false, having written nothing, when the graph cannot be
// taken (16-bit ids, edge capacity, shared memory); every CTA returns the same.
template <int C>
__device__ bool cl_solve(const DevScene &ds, int max_rounds, cg::cluster_group &cluster, ClShared &sh,
                         unsigned char *sm_raw) {
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = kClThreads / 32;
#ifdef SPM_COUNT
    const long long t_cl0 = clock64();
#endif
    const int n = ds.n_gen, nv = ds.n_vert, ns = ds.n_src;
    if (nv == 0) {  // sources only: nothing to relax
        if (rank == 0) {
            for (int g = tid; g < ns; g += kClThreads) {
                ds.cost[0][g] = 0.0;
                ds.par[0][g] = g;
                ds.gen_cone[g] = make_int4(0, 0, 0, 0);
                ds.gen_ctype[g] = kConeNone;
                finalize_gen(ds, g, 0.0, g);
            }
            if (tid == 0) ds.stats[0] = 0;
        }
        return true;
    }
    const long long E = ds.in_start[nv];
    if (n >= 32768 || E > ds.edge_cap) return false;
    static_assert(C <= kClGrp, "a changed vertex's group writes every CTA's copy");
    const int nmax = (nv + C - 1) / C;
    const int n_own = rank < nv ? (nv - rank + C - 1) / C : 0;  // vertices vv = rank + C * k
    // the state and the offset arrays sit at offsets that do not depend on
    // the in-list sizes; when even they do not fit, nothing does
    const ClLayout L0 = cl_layout(n, nv, 0, false, C);
    if (L0.lin_src > (size_t)kClSmem) return false;
    // every CTA's in-edge count, in each CTA (warp r sums CTA r's vertices):
    // the largest decides the layout, the same in all, with no exchange
    if (warp < C) {
        long long m = 0;
        for (int vv = warp + C * lane; vv < nv; vv += 32 * C) m += ds.in_start[vv + 1] - ds.in_start[vv];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
        if (lane == 0) sh.own_e[warp] = m;
    }
    // this CTA's in-list offsets: a scan over its vertices, in chunks, with
    // their global starts kept
    int *gstart = (int *)(sm_raw + L0.gstart);
    const int per = (n_own + kClThreads - 1) / kClThreads, lo = min(n_own, tid * per), hi = min(n_own, lo + per);
    long long mine = 0;
    int *lin_start = (int *)(sm_raw + L0.lin_start);
    for (int k = lo; k < hi; ++k) {
        const int a = ds.in_start[rank + C * k], d = ds.in_start[rank + C * k + 1] - a;
        gstart[k] = a;
        lin_start[k] = d;  // the degree, until the offsets replace it
        mine += d;
    }
    const long long before = cta_exclusive_scan(mine, sh.wsum);  // its barriers publish own_e too
    long long mx = 0;
    for (int r = 0; r < C; ++r) mx = max(mx, sh.own_e[r]);
    const int fit = cl_layout(n, nv, mx, true, C).end <= (size_t)kClSmem ? 2 : cl_layout(n, nv, mx, false, C).end <= (size_t)kClSmem ? 1 : 0;
    if (!fit) return false;
    const bool with_len = fit == 2;
    const ClLayout L = cl_layout(n, nv, sh.own_e[rank], with_len, C);
    double *cost = (double *)(sm_raw + L.cost);
    short4 *wedge = (short4 *)(sm_raw + L.wedge);
    short *par = (short *)(sm_raw + L.par);
    short2 *lat = (short2 *)(sm_raw + L.lat);
    short4 *ldir = (short4 *)(sm_raw + L.ldir);                // lattice position, arrival direction from the parent
    unsigned *chg = (unsigned *)(sm_raw + L.chg);              // changed generators, round parity p at p * cw
    unsigned short *dl = (unsigned short *)(sm_raw + L.dl);    // round parity p at p * nmax
    unsigned short *lin_src = (unsigned short *)(sm_raw + L.lin_src);
    double *lin_len = (double *)(sm_raw + L.lin_len);          // with_len only
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    {
        long long run = before;
        for (int k = lo; k < hi; ++k) {
            const int d = lin_start[k];
            lin_start[k] = (int)run;
            run += d;
        }
        if (hi == n_own && lo < hi) lin_start[n_own] = (int)run;
        if (tid == 0 && n_own == 0) lin_start[0] = 0;
    }
    for (int g = tid; g < n; g += kClThreads) {
        const bool src = g < ns;
        cost[g] = ds.warm ? ds.warm_cost[g] : src ? 0.0 : inf;  // warm: the tree's state
        par[g] = (short)(ds.warm ? ds.warm_par[g] : src ? g : -1);
        const int2 l = ds.gen_lat[g];
        lat[g] = make_short2((short)l.x, (short)l.y);
        const int4 w = ds.gen_wedge[g];
        wedge[g] = make_short4((short)w.x, (short)w.y, (short)w.z, (short)w.w);
    }
    for (int w = tid; w < 2 * ((n + 31) / 32); w += kClThreads) chg[w] = 0u;
    for (int g = tid; g < min(ns, kSoloSrc); g += kClThreads) {
        const int k = ds.gen_kind[g];
        sh.src_kind[g] = (signed char)k;
        sh.src_seg[g] = k == kSegI ? ds.seg_lat[ds.gen_aux[g]] : make_int4(0, 0, 0, 0);
    }
    if (tid < 3) sh.cnt[tid] = 0;
    __syncthreads();  // lin_start, lat, par, the sources' segments
    // each generator's arrival direction from its parent ((0, 0) while it
    // has none: no shadow cone then holds it)
    for (int g = tid; g < n; g += kClThreads) {
        const int p = par[g];
        int dx = 0, dy = 0;
        if (p >= 0) arrival_from(ds, sh.src_kind, sh.src_seg, lat, p, lat[g], dx, dy);
        ldir[g] = make_short4(lat[g].x, lat[g].y, (short)dx, (short)dy);
    }
    for (int k = warp; k < n_own; k += nwarps) {  // this CTA's in-lists, a warp per vertex
        const int e0 = gstart[k], b = lin_start[k], m = lin_start[k + 1] - b;
        for (int j = lane; j < m; j += 32) {
            lin_src[b + j] = (unsigned short)ds.in_src[e0 + j];
            if (with_len) lin_len[b + j] = ds.in_len[e0 + j];
        }
    }
    cluster.sync();  // every CTA's bitmaps and counts are ready for marks
    constexpr int kGpw = 32 / kClGrp;
    const int grp = lane / kClGrp, gl = lane % kClGrp, ngroups = nwarps * kGpw;
    const unsigned kFull = 0xffffffffu;
    // A round's changes are broadcast as bits: a changed vertex sets its bit
    // in every CTA's bitmap of the round's parity (remote ORs whose result
    // nobody waits for), so after the cluster barrier every CTA holds the
    // same set of changed generators and finds its own dirty vertices --
    // those with a changed in-neighbour -- by scanning its in-lists locally.
    const int cw = (n + 31) / 32;
    if (ds.warm) {  // round 0 pulls the vertices whose equation the tree's state breaks; each CTA its own
        const int m = min(ds.counters[6], nv);
        for (int i = tid; i < m; i += kClThreads) {
            const int vv = ds.dirtyl[0][i] - ns;
            if (vv % C == rank) dl[atomicAdd(&sh.cnt[0], 1)] = (unsigned short)(vv / C);
        }
    } else {  // round 0 pulls the vertices with a source in-neighbour: the sources count as changed
        for (int g = tid; g < ns; g += kClThreads) atomicOr(&chg[g >> 5], 1u << (g & 31));
    }
    __syncthreads();
#ifdef SPM_COUNT
    const long long t_cl1 = clock64();
    if (rank == 0 && tid == 0) SPM_CNT(17, t_cl1 - t_cl0);  // prologue: layout checks, state and in-lists staged
#endif
    int round = 0;
    for (;; ++round) {
        const int cur = round & 1, nxt = cur ^ 1;
        unsigned *chc = chg + cur * cw;  // changed in the last round (the same bits in every CTA)
        if (round > 0 || !ds.warm) {
            int any = 0;
            for (int w = tid; w < cw; w += kClThreads) any |= chc[w] != 0u;
            if (!__syncthreads_or(any)) break;  // no change anywhere: every CTA stops here
            if (round >= max_rounds) {
                if (rank == 0 && tid == 0) atomicOr(ds.status, kStNotConverged);
                break;
            }
#ifdef SPM_COUNT
            const long long t_r0 = clock64();
#endif
            for (int k0 = warp * kGpw; k0 < n_own; k0 += ngroups) {  // warp-uniform trip count
                const int k = k0 + grp;
                bool hit = false;
                if (k < n_own)
                    for (int e = lin_start[k] + gl, e1 = lin_start[k + 1]; e < e1 && !hit; e += kClGrp) {
                        const int u = lin_src[e];
                        hit = (chc[u >> 5] >> (u & 31)) & 1u;
                    }
                const unsigned bal = __ballot_sync(kFull, hit);
                if (gl == 0 && ((bal >> (grp * kClGrp)) & ((1u << kClGrp) - 1u)))
                    dl[cur * nmax + atomicAdd(&sh.cnt[cur], 1)] = (unsigned short)k;
            }
            __syncthreads();
#ifdef SPM_COUNT
            if (rank == 0 && tid == 0) SPM_CNT(20, clock64() - t_r0);  // finding the dirty vertices
#endif
            // read: free again (this round's changes go to the other parity)
            for (int w = tid; w < cw; w += kClThreads) chc[w] = 0u;
        }
        const int nd = sh.cnt[cur];
#ifdef SPM_COUNT
        const long long t_p0 = clock64();
        if (rank == 0 && tid == 0) SPM_CNT(22, nd);
#endif
        for (int i0 = warp * kGpw; i0 < nd; i0 += ngroups) {  // warp-uniform trip count
            const int i = i0 + grp;
            const bool act = i < nd;
            const int lw = dl[cur * nmax + min(i, nmax - 1)];
            const int lk = act ? lw : 0;
            const int vv = rank + C * lk, v = ns + vv;
            const int e0 = lin_start[lk] + gl, e1 = act ? lin_start[lk + 1] : 0;
            const int eg = gstart[lk] - lin_start[lk];  // local -> global edge index (lengths)
            const short2 vl = lat[v];
            const long long cv = __double_as_longlong(cost[v]);
            const int pv = par[v];
            long long best = 0x7ff0000000000000ll;  // +inf bits
            int bpar = -1;
            for (int e = e0; e < e1; e += kClGrp) {
                const double len = with_len ? lin_len[e] : __ldg(ds.in_len + eg + e);
                const int u = lin_src[e];
                const double cu = cost[u];
                const short4 q = ldir[u];  // u's position and arrival direction
                const short4 w = wedge[u];
                const bool valid = (__double_as_longlong(cu) < 0x7ff0000000000000ll) &
                                   ((u < ns) | in_shadow_cone(q.z, q.w, w, vl.x - q.x, vl.y - q.y));
                const long long cand = __double_as_longlong(__dadd_rn(cu, len));
                const bool better = valid & (cand < best);
                best = better ? cand : best;
                bpar = better ? u : bpar;
            }
#pragma unroll
            for (int o = kClGrp / 2; o > 0; o >>= 1) {  // within the group
                const long long ob = __shfl_xor_sync(kFull, best, o);
                const int op = __shfl_xor_sync(kFull, bpar, o);
                if (ob < best || (ob == best && (unsigned)op < (unsigned)bpar)) {
                    best = ob;
                    bpar = op;
                }
            }
            const bool changed = act && (best != cv || bpar != pv);
            if (changed && gl < C) {  // lane gl writes CTA gl's copy and its changed bit
                int dx = 0, dy = 0;
                if (bpar >= 0) arrival_from(ds, sh.src_kind, sh.src_seg, lat, bpar, vl, dx, dy);
                cluster.map_shared_rank(cost, gl)[v] = __longlong_as_double(best);
                cluster.map_shared_rank(par, gl)[v] = (short)bpar;
                cluster.map_shared_rank(ldir, gl)[v] = make_short4(vl.x, vl.y, (short)dx, (short)dy);
                atomicOr(cluster.map_shared_rank(chg, gl) + nxt * cw + (v >> 5), 1u << (v & 31));
            }
        }
        if (tid == 0) sh.cnt[nxt] = 0;  // the next round's list (last read two rounds ago)
#ifdef SPM_COUNT
        __syncthreads();
        const long long t_p1 = clock64();
        if (rank == 0 && tid == 0) SPM_CNT(21, t_p1 - t_p0);  // the pulls
#endif
        cluster.sync();
#ifdef SPM_COUNT
        if (rank == 0 && tid == 0) SPM_CNT(23, clock64() - t_p1);  // the cluster barrier
#endif
    }
#ifdef SPM_COUNT
    if (rank == 0 && tid == 0) {
        SPM_CNT(18, clock64() - t_cl1);  // the rounds
        SPM_CNT(19, round);
    }
#endif
    cluster.sync();  // the last round's remote reads of the counts are done
    // the settled state of this CTA's vertices (and, in CTA 0, the sources),
    // with each vertex's shadow cone from its parent
    for (int k = tid; k < n_own + (rank == 0 ? ns : 0); k += kClThreads) {
        const int g = k < n_own ? ns + rank + C * k : k - n_own;
        const int pg = par[g];
        int4 c = make_int4(0, 0, 0, 0);
        int ct = kConeNone;
        if (g >= ns) {
            ct = kConeEmpty;
            if (pg >= 0) {
                int dx, dy;
                arrival_from(ds, sh.src_kind, sh.src_seg, lat, pg, lat[g], dx, dy);
                const short4 w = wedge[g];
                ct = make_cone(make_int4(w.x, w.y, w.z, w.w), dx, dy, c);
            }
        }
        ds.cost[0][g] = cost[g];
        ds.par[0][g] = pg;
        ds.gen_cone[g] = c;
        ds.gen_ctype[g] = ct;
        finalize_gen(ds, g, cost[g], pg);
    }
    if (rank == 0 && tid == 0) ds.stats[0] = round;
    cluster.sync();  // this scene's shared memory is no longer read
    return true;
}

template <int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kClThreads)
    k_sssp_cluster(const __grid_constant__ DevScene ds, int max_rounds) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    chain_start();
    __shared__ ClShared sh;
    cg::cluster_group cluster = cg::this_cluster();
    bool solo_len;
    if (solo_bytes(ds, solo_len) > 0) return;  // the single-CTA kernel handles this graph (every CTA agrees)
    const bool done = cl_solve<C>(ds, max_rounds, cluster, sh, sm_raw);
    if (cluster.block_rank() == 0 && threadIdx.x == 0) ds.counters[4] = done ? 1 : 0;  // else the many-CTA kernel
}

// Batched form: resident clusters take the batch's scenes from a counter,
// most generators first, each solving one scene's fixpoint at a time; a
// scene one cluster cannot take is left to the many-CTA batched kernel.
__global__ void __cluster_dims__(kClCtas, 1, 1) __launch_bounds__(kClThreads)
    k_sssp_cluster_b(const __grid_constant__ BatchDev b) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ ClShared sh;
    cg::cluster_group cluster = cg::this_cluster();
    const bool lead = cluster.block_rank() == 0 && threadIdx.x == 0;
    for (;;) {
        if (lead) sh.next = atomicAdd(b.cl_counter, 1);
        cluster.sync();
        const int k = *cluster.map_shared_rank(&sh.next, 0);
        cluster.sync();  // every CTA has read it before the next is taken
        if (k >= b.n) break;
        const int sc = b.cl_order[k];
        const bool done = cl_solve<kClCtas>(b.scenes[sc], b.max_rounds, cluster, sh, sm_raw);
        if (lead) b.cl_done[sc] = done ? 1 : 0;
    }
}

// Final generator table for the pixel phase: FP32 costs and shadow cones.
// After the many-CTA fixpoint (the single-CTA and cluster kernels finalise
// their own results).
__global__ void k_finalize(const __grid_constant__ DevScene ds) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ds.n_gen; g += gridDim.x * blockDim.x)
        finalize_gen(ds, g, ds.cost[0][g], ds.par[0][g]);
}

// ---------------------------------------------------------------------------
// Batched forms: the same per-scene work for every scene of a batch in one
// launch per step. Global task indices map to (scene, local index) through
// prefix offsets (binary search over scenes).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ int scene_of(const T *off, int n, T x) {
    int lo = 0, hi = n;  // last scene with off[s] <= x
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_prepare_b(const __grid_constant__ BatchDev b) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.vert_off[b.n]; i += gridDim.x * blockDim.x) {
        // every scene's bit matrix, a row per thread: with kept edge lists
        // only the source columns are read, and they start empty; else the
        // row's static part
        const int s = scene_of(b.vert_off, b.n, i);
        const DevScene &ds = b.scenes[s];
        uint32_t *row = ds.vis_bits + (size_t)(i - b.vert_off[s]) * ds.vis_words;
        const uint32_t *srow = ds.vis_static ? ds.vis_static + (size_t)(i - b.vert_off[s]) * ds.vis_words : nullptr;
        const int nw = ds.st_start ? (ds.n_src + 31) / 32 : ds.vis_words;
        for (int w = 0; w < nw; ++w) row[w] = srow && !ds.st_start ? srow[w] : 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *reinterpret_cast<unsigned long long *>(b.counters + 6) = 0ull;  // visibility-pair work counter
    const int total = b.gen_off[b.n];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total + b.n; i += gridDim.x * blockDim.x) {
        // entries 0..total-1: one per generator; total..total+n-1: one per scene
        if (i < total) {
            const int s = scene_of(b.gen_off, b.n, i);
            const DevScene &ds = b.scenes[s];
            const int g = i - b.gen_off[s];
            ds.out_start[g + 1] = ds.st_out_init ? ds.st_out_init[g + 1] : 0;
            ds.out_fill[g] = 0;
        } else {
            const DevScene &ds = b.scenes[i - total];
            ds.out_start[0] = 0;
            if (ds.n_vert == 0) ds.in_start[0] = 0;
        }
    }
}

__global__ void __launch_bounds__(kVisThreads) k_vis_pairs_b(const __grid_constant__ BatchDev b) {
    __shared__ PairQ q;
    vis_pairs_run(
        q, b.pair_off[b.n], 4, reinterpret_cast<unsigned long long *>(b.counters + 6), [&](int s) { return b.scenes + s; },
        [&](long long t, int &sc, long long &lt) {
            sc = scene_of(b.pair_off, b.n, t);
            lt = t - b.pair_off[sc];
        });
}

__global__ void k_edges_count_b(const __grid_constant__ BatchDev b) {
    const int lane = threadIdx.x & 31, nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < b.vert_off[b.n]; i += nw) {
        const int s = scene_of(b.vert_off, b.n, i);
        edges_count_row(b.scenes[s], i - b.vert_off[s], lane);
    }
}

__global__ void __launch_bounds__(1024) k_edges_scan_b(const __grid_constant__ BatchDev b) {
    __shared__ long long part[32];
    const DevScene &ds = b.scenes[blockIdx.x];
    if (ds.n_vert > 0) edges_scan_block(ds, part);
}

__global__ void k_edges_fill_b(const __grid_constant__ BatchDev b) {
    const int lane = threadIdx.x & 31, nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < b.vert_off[b.n]; i += nw) {
        const int s = scene_of(b.vert_off, b.n, i);
        const DevScene &ds = b.scenes[s];
        if (ds.in_start[ds.n_vert] > ds.edge_cap) continue;
        edges_fill_row(ds, i - b.vert_off[s], lane);
        if (ds.st_start) edges_out_copy(ds, i - b.vert_off[s], lane);  // vertex i's kept out-list
    }
}

__device__ __forceinline__ void mark_out_warp_b(const DevScene &ds, int s, int u, int lane, int2 *dl,
                                                int32_t *dcount) {
    const int e0 = ds.out_start[u], e1 = ds.out_start[u + 1];
    for (int eb = e0; eb < e1; eb += 32) {
        const int e = eb + lane;
        bool fresh = false;
        int v = 0;
        if (e < e1) {
            v = ds.out_dst[e];
            const uint32_t bit = 1u << (v & 31);
            fresh = !(atomicOr(&ds.dirty[v >> 5], bit) & bit);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, fresh);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(dcount, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (fresh) dl[base + __popc(bal & ((1u << lane) - 1u))] = make_int2(s, v);
    }
}

// The cooperative fixpoint of k_sssp over every scene at once: dirty and
// changed lists hold (scene, vertex) entries, rounds run until no scene
// changes (the deepest scene sets the round count).
__global__ void __launch_bounds__(256) k_sssp_b(const __grid_constant__ BatchDev b) {
    cg::grid_group grid = cg::this_grid();
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsize = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, gwarp = gtid >> 5, nwarps = gsize >> 5;
    int32_t *cnt = b.counters;
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    const int total = b.gen_off[b.n];
    for (int i = gtid; i < total; i += gsize) {
        const int s = scene_of(b.gen_off, b.n, i);
        if (b.cl_done[s]) continue;  // a cluster solved this scene
        const DevScene &ds = b.scenes[s];
        const int g = i - b.gen_off[s];
        const bool src = g < ds.n_src;
        ds.cost[0][g] = src ? 0.0 : inf;
        ds.par[0][g] = src ? g : -1;
        ds.gen_ctype[g] = src ? kConeNone : kConeEmpty;
        ds.gen_cone[g] = make_int4(0, 0, 0, 0);
        if ((g & 31) == 0) ds.dirty[g >> 5] = 0u;
    }
    if (gtid < 5) cnt[gtid] = 0;
    grid.sync();
    for (int i = gwarp; i < total; i += nwarps) {  // sources mark their out-neighbours
        const int s = scene_of(b.gen_off, b.n, i);
        const DevScene &ds = b.scenes[s];
        const int g = i - b.gen_off[s];
        if (g < ds.n_src && !b.cl_done[s] && ds.in_start[ds.n_vert] <= ds.edge_cap)
            mark_out_warp_b(ds, s, g, lane, b.dirtyl[0], &cnt[2]);
    }
    grid.sync();
    int round = 0;
    for (;; ++round) {
        const int par_r = round & 1, par_n = par_r ^ 1;
        if (gtid == 0) {
            cnt[par_n] = 0;
            cnt[2 + par_n] = 0;
        }
        const int nd = __ldcg(&cnt[2 + par_r]);
        for (int i = gwarp; i < nd; i += nwarps) {
            const int2 ent = __ldcg(&b.dirtyl[par_r][i]);
            const int s = ent.x, v = ent.y;
            const DevScene &ds = b.scenes[s];
            const int vv = v - ds.n_src;
            if (lane == 0) atomicAnd(&ds.dirty[v >> 5], ~(1u << (v & 31)));
            const int2 vl = ds.gen_lat[v];
            long long best = 0x7ff0000000000000ll;
            int bpar = -1;
            for (int e = ds.in_start[vv] + lane; e < ds.in_start[vv + 1]; e += 32) {
                const int u = ds.in_src[e];
                const double cu = __ldcg(&ds.cost[0][u]);
                if (__double_as_longlong(cu) >= 0x7ff0000000000000ll) continue;
                const int ct = __ldcg(&ds.gen_ctype[u]);
                if (ct != kConeNone) {
                    const int2 ul = ds.gen_lat[u];
                    if (!in_cone(ct, __ldcg(&ds.gen_cone[u]), vl.x - ul.x, vl.y - ul.y)) continue;
                }
                const long long cand = __double_as_longlong(__dadd_rn(cu, ds.in_len[e]));
                if (cand < best || (cand == best && u < bpar)) {
                    best = cand;
                    bpar = u;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int op = __shfl_xor_sync(0xffffffffu, bpar, o);
                if (ob < best || (ob == best && (unsigned)op < (unsigned)bpar)) {
                    best = ob;
                    bpar = op;
                }
            }
            if (lane == 0 && (best != __double_as_longlong(__ldcg(&ds.cost[0][v])) || bpar != __ldcg(&ds.par[0][v]))) {
                ds.cost[1][v] = __longlong_as_double(best);
                ds.par[1][v] = bpar;
                b.frontier[par_r][atomicAdd(&cnt[par_r], 1)] = make_int2(s, v);
            }
        }
        grid.sync();
        const int nc = __ldcg(&cnt[par_r]);
        if (nc == 0) break;
        if (round + 1 >= b.max_rounds) {
            if (gtid == 0) cnt[4] = -1;
            break;
        }
        for (int i = gtid; i < nc; i += gsize) {
            const int2 ent = __ldcg(&b.frontier[par_r][i]);
            commit_vertex(b.scenes[ent.x], ent.y);
        }
        for (int i = gwarp; i < nc; i += nwarps) {
            const int2 ent = __ldcg(&b.frontier[par_r][i]);
            mark_out_warp_b(b.scenes[ent.x], ent.x, ent.y, lane, b.dirtyl[par_n], &cnt[2 + par_n]);
        }
        grid.sync();
    }
    for (int s = gtid; s < b.n; s += gsize) {
        if (b.cl_done[s]) continue;
        const DevScene &ds = b.scenes[s];
        ds.stats[0] = round + 1;
        if (cnt[4] < 0) atomicOr(ds.status, kStNotConverged);
    }
}

__global__ void k_finalize_b(const __grid_constant__ BatchDev b) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.gen_off[b.n]; i += gridDim.x * blockDim.x) {
        const int s = scene_of(b.gen_off, b.n, i);
        {
            const DevScene &d = b.scenes[s];
            const int g = i - b.gen_off[s];
            finalize_gen(d, g, d.cost[0][g], d.par[0][g]);
        }
    }
}

}  // namespace

int vis_resident_blocks();  // co-resident CTAs of the visibility-pair kernel

// Round cap of the vertex fixpoint: 4 rounds per generator and 64 more (far
// above the longest shortest path in links), or the test hook's override.
std::atomic<int> g_round_cap_override{0};
std::atomic<int> g_many_cta_override{0};
int fixpoint_round_cap(int n_gen) {
    const int o = g_round_cap_override.load();
    return o > 0 ? o : 4 * n_gen + 64;
}

// Visibility-pair kernel over ds's pair range (resident CTAs, runs sized so
// that every resident warp takes about two).
// The start values of a compute's vertex phase, in one launch: out-degrees
// (the kept obstacle vertices', or zero), fill cursors, the source columns of
// the bit matrix (with kept edge lists), the pair kernel's work counter, the
// cluster kernel's done flag and, for a warm start, the estimates (a huge
// value: none yet) and the count of unsatisfied vertices.
__global__ void k_vertex_prep(const __grid_constant__ DevScene ds) {
    chain_start();
    const int sw = (ds.n_src + 31) / 32;
    const long long n_bits = ds.st_start ? (long long)ds.n_vert * sw : 0;
    const long long items = max((long long)ds.n_gen + 1, n_bits);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < items; i += (long long)gridDim.x * blockDim.x) {
        if (i <= ds.n_gen) ds.out_start[i] = ds.st_out_init ? ds.st_out_init[i] : 0;
        if (i < ds.n_gen) ds.out_fill[i] = 0;
        if (i < n_bits) ds.vis_bits[(i / sw) * ds.vis_words + i % sw] = 0u;
        if (ds.warm && i < ds.n_vert) ds.warm_est[i] = __longlong_as_double(0x7f7f7f7f7f7f7f7fll);  // 1.4e306
        if (i == 0) {
            *reinterpret_cast<unsigned long long *>(ds.stats + 2) = 0ull;  // the pair kernel's work counter
            ds.counters[4] = 0;
            ds.counters[6] = 0;
        }
    }
}

// Launches a kernel of the vertex phase's chain with programmatic stream
// serialization (it may be scheduled while its predecessor runs and waits
// for it in chain_start); an ordinary launch if the attribute is refused.
template <typename... KArgs, typename... Args>
static void launch_chained(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                           Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, args...) != cudaSuccess) {
        cudaGetLastError();
        kern<<<grid, block, smem, st>>>(args...);
    }
}

void launch_pairs(const DevScene &ds, cudaStream_t st, bool reset_counter = true) {
    const long long tasks = (long long)ds.n_vert * ds.pair_words;
    if (reset_counter) cudaMemsetAsync(ds.stats + 2, 0, sizeof(unsigned long long), st);  // the pair kernel's work counter
    if (tasks == 0) return;
    const int resident = vis_resident_blocks();
    long long blocks = (tasks + (kVisThreads / 32) - 1) / (kVisThreads / 32);  // a task per warp at least
    blocks = blocks > resident ? resident : blocks;
    const long long per_chunk = tasks / (blocks * (kVisThreads / 32) * 2);
    const int chunk = (int)(per_chunk < 1 ? 1 : (per_chunk > 32 ? 32 : per_chunk));
    launch_chained(k_vis_pairs, dim3((int)blocks), dim3(kVisThreads), 0, st, ds, chunk);
}

void launch_vis_static(const DevScene &ds, cudaStream_t st, uint32_t *vis_static) {
    if (ds.n_vert == 0) return;
    cudaMemsetAsync(vis_static, 0, sizeof(uint32_t) * (size_t)ds.n_vert * ds.vis_words, st);
    DevScene d = ds;  // every word of every row, obstacle-vertex columns only
    d.vis_bits = vis_static;
    d.vis_static = nullptr;
    d.pair_words = ds.vis_words;
    d.pair_u0 = ds.n_src;
    d.pair_u1 = ds.n_gen;
    launch_pairs(d, st);
}


// Which fixpoint kernels a compute launches. A vertex's in-edges are its
// obstacle-vertex pairs in the scene's static bits, fixed, plus at most one
// from each source; those bounds decide, per kernel, whether it surely takes
// every compute's graph, surely takes none, or has to see the graph.
int fixpoint_launches(const DevScene &ds, const std::vector<int32_t> &deg) {
    int f = (ds.solo_smem > 0 ? kFixSolo : 0) | (cluster_smem_ok() ? kFixCluster : 0);
    const int nv = ds.n_vert;
    if ((int)deg.size() < nv) return f;  // unknown: the kernels decide on the device
    // the most in-edges one CTA of a C-CTA cluster holds (vertices dealt round-robin)
    auto own_max = [&](int C) {
        long long m = 0;
        for (int r = 0; r < C; ++r) {
            long long own = 0;
            for (int vv = r; vv < nv; vv += C) own += deg[vv] + ds.n_src;
            m = std::max(m, own);
        }
        return m;
    };
    long long lo = 0;
    for (int vv = 0; vv < nv; ++vv) lo += deg[vv];
    const long long hi = lo + (long long)ds.n_src * nv;
    // the single-CTA kernel's test only gets stricter as the edges grow
    bool wl;
    const bool solo_never = solo_bytes_for(ds.n_gen, nv, lo, ds.edge_cap, ds.solo_smem, wl) == 0;
    const bool solo_sure = solo_bytes_for(ds.n_gen, nv, hi, ds.edge_cap, ds.solo_smem, wl) > 0;
    if (solo_never) f &= ~kFixSolo;
    // Beside a single-CTA launch the cluster kernel only stands by (it
    // returns when the single-CTA kernel took the graph). As that kernel's
    // dependent launch it is resident while the other runs and holds its
    // SMs, which the sources' culling on the side stream would use: it takes
    // the portable size there.
    const int C = (f & kFixSolo) && !solo_sure ? kClCtas : cluster_ctas();
    const bool cluster_ok = (f & kFixCluster) && ds.n_gen < 32768 && hi <= ds.edge_cap;
    const bool cluster_sure = cluster_ok && cl_layout(ds.n_gen, nv, own_max(C), false, C).end <= (size_t)kClSmem;
    if (C == kClCtasWide) f |= kFixClusterWide;
    // the batched form's clusters are of the portable size
    if (cluster_ok && cl_layout(ds.n_gen, nv, own_max(kClCtas), false, kClCtas).end <= (size_t)kClSmem)
        f |= kFixClusterFits;
    if (solo_sure) f = (f & ~kFixCluster) | kFixSoloSure;
    if (cluster_sure && !solo_sure) f |= kFixClusterSure;
    return f;
}

void launch_static_lengths(const DevScene &ds, double *len, cudaStream_t st) {
    if (ds.n_vert > 0) k_static_lengths<<<std::min((ds.n_vert + 7) / 8, 152 * 8), 256, 0, st>>>(ds, len);
}

// The GPU can hold at least one cluster of C CTAs of the kernel.
static bool cluster_holds(const void *kern, int C) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = kClSmem;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return clusters > 0;
}

// The single-scene cluster fixpoint's CTAs: 16 (a non-portable cluster
// size, twice the SMs a round) where the GPU holds such a cluster, else the
// portable 8, 0 when neither can run. Shared memory is granted once per
// process, to the batched kernel too.
int cluster_ctas() {
    static const int ctas = [] {
        const void *k16 = (const void *)k_sssp_cluster<kClCtasWide>, *k8 = (const void *)k_sssp_cluster<kClCtas>;
        if (cudaFuncSetAttribute(k8, cudaFuncAttributeMaxDynamicSharedMemorySize, kClSmem) != cudaSuccess ||
            cudaFuncSetAttribute((const void *)k_sssp_cluster_b, cudaFuncAttributeMaxDynamicSharedMemorySize, kClSmem) !=
                cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        if (cudaFuncSetAttribute(k16, cudaFuncAttributeMaxDynamicSharedMemorySize, kClSmem) == cudaSuccess &&
            cudaFuncSetAttribute(k16, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
            cluster_holds(k16, kClCtasWide))
            return kClCtasWide;
        cudaGetLastError();
        return cluster_holds(k8, kClCtas) ? kClCtas : 0;
    }();
    return ctas;
}

bool cluster_smem_ok() { return cluster_ctas() > 0; }

// ---------------------------------------------------------------------------
// Warm start of the fixpoint. Obstacles never move, so the geodesic
// distances between obstacle vertices over the kept obstacle-vertex edges
// are computed once per scene (k_vtab_build). A compute then
//   k_warm_entry: estimates each obstacle vertex's cost as the least
//       m(u) + tab(u, v) over the vertices u a source links to, m(u) being
//       u's shortest source link;
//   k_warm_tree:  picks for each vertex the in-neighbour u with the least
//       estimate(u) + |u - v| (sources estimate 0), the tree parent;
//   k_warm_fold:  evaluates the FP64 cost along that tree as the fixpoint
//       accumulates it, cost(v) = cost(parent) + |parent - v|, from the
//       sources down (depths by pointer doubling, a counting sort by depth,
//       one warp folding level by level);
//   k_warm_verify: lists the vertices whose equation that state breaks
//       (the fixpoint's pull gives another cost or parent);
// and the fixpoint kernels start from that state with those vertices dirty.
// The fixpoint of the vertex equations is unique, so the result is the
// cold start's bit for bit; the tree only spares the rounds in which a start
// from the sources alone carries costs down long chains of links (one round
// a link). Where the tree is wrong (near ties of the estimates, cones) the
// rounds that follow correct it.

constexpr int kVtabWarps = 4;  // roots in flight per CTA of the table build
constexpr double kEstNone = 1e300;  // estimates at or above this mean "not reached"

__host__ __device__ __forceinline__ size_t vtab_list_bytes(int nv) { return ((size_t)4 * nv + 15) & ~(size_t)15; }
__host__ __device__ __forceinline__ size_t vtab_warp_bytes(int nv) {
    return vtab_list_bytes(nv) + ((((size_t)nv + 31) / 32 * 4 + 15) & ~(size_t)15);
}

// One warp per root vertex r, roots taken from a counter: Bellman-Ford rounds
// over the kept edges, the frontier pushing cost(u) + |u - w| into row r by
// 64-bit atomic minima (non-negative doubles order like their bit patterns).
// The kept lists are symmetric between obstacle vertices (each pair is tested
// once and its edge mirrored), so a vertex's in-list is its out-list. The
// table only guides the start: any order of the sums will do.
__global__ void __launch_bounds__(32 * kVtabWarps) k_vtab_build(const __grid_constant__ DevScene ds, double *tab,
                                                                int32_t *counter) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ int cnt[kVtabWarps];
    const int nv = ds.n_vert, ns = ds.n_src, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int dw = (nv + 31) / 32;
    unsigned char *base = sm_raw + (size_t)warp * vtab_warp_bytes(nv);
    unsigned short *list = (unsigned short *)base;                  // two lists of nv entries, by round parity
    unsigned *inl = (unsigned *)(base + vtab_list_bytes(nv));       // vertex already in the next list
    const unsigned kFull = 0xffffffffu;
    const unsigned long long kInfBits = 0x7ff0000000000000ull;
    for (;;) {
        int r = 0;
        if (lane == 0) r = atomicAdd(counter, 1);
        r = __shfl_sync(kFull, r, 0);
        if (r >= nv) return;
        unsigned long long *row = (unsigned long long *)(tab + (size_t)r * nv);
        for (int v = lane; v < nv; v += 32) row[v] = v == r ? 0ull : kInfBits;
        for (int w = lane; w < dw; w += 32) inl[w] = 0u;
        if (lane == 0) list[0] = (unsigned short)r;
        int nc = 1, cur = 0;
        __syncwarp();
        for (int round = 0; nc > 0 && round <= nv; ++round) {
            const int nxt = cur ^ 1;
            if (lane == 0) cnt[warp] = 0;
            for (int i = lane; i < nc; i += 32) {  // the members of this list may enter the next one again
                const int u = list[cur * nv + i];
                atomicAnd(&inl[u >> 5], ~(1u << (u & 31)));
            }
            __syncwarp();
            for (int i = lane; i < nc; i += 32) {
                const int u = list[cur * nv + i];
                const double cu = __longlong_as_double((long long)__ldcg(row + u));  // minima land in L2
                const int e1 = __ldg(ds.st_start + u + 1);
                for (int e = __ldg(ds.st_start + u); e < e1; ++e) {
                    const int w = __ldg(ds.st_src + e) - ns;
                    const unsigned long long nd = (unsigned long long)__double_as_longlong(__dadd_rn(cu, __ldg(ds.st_len + e)));
                    if (nd < atomicMin(row + w, nd)) {
                        const unsigned bit = 1u << (w & 31);
                        if (!(atomicOr(&inl[w >> 5], bit) & bit)) list[nxt * nv + atomicAdd(&cnt[warp], 1)] = (unsigned short)w;
                    }
                }
            }
            __syncwarp();
            nc = cnt[warp];
            cur = nxt;
            __syncwarp();  // every lane has the count before lane 0 clears it
            if (nc == 0 && lane == 0) atomicMax(counter + 1, round + 1);  // the deepest root's rounds
        }
    }
}

// Estimated cost of each obstacle vertex v: the least m(u) + tab(u, v) over
// the vertices u with a source link, m(u) the shortest of them (a compute's
// in-list of u starts with its source links: sources have the smallest
// generator ids). Adding a length rounds monotonically, so taking m(u) first
// loses nothing. Grid: x over 256 targets v, y over 128 candidate vertices u;
// each CTA folds its share into warm_est (preset to a huge value) by 64-bit
// atomic minima.
constexpr int kEntryRows = 128;
__global__ void __launch_bounds__(256) k_warm_entry(const __grid_constant__ DevScene ds) {
    chain_start();
    __shared__ int eu[kEntryRows];
    __shared__ double em[kEntryRows];
    __shared__ int ne;
    const int nv = ds.n_vert, ns = ds.n_src, tid = threadIdx.x;
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    if (tid == 0) ne = 0;
    __syncthreads();
    if (tid < kEntryRows) {
        const int u = blockIdx.y * kEntryRows + tid;
        if (u < nv) {
            // u's source links, from the source columns of its bit row (the
            // edge lists need not be built yet)
            double m = inf;
            const uint32_t *row = ds.vis_bits + (size_t)u * ds.vis_words;
            for (int w = 0; w * 32 < ns; ++w)
                for (uint32_t b = row[w] & src_word_mask(ds, w); b; b &= b - 1)
                    m = fmin(m, edge_len(ds, w * 32 + __ffs(b) - 1, ns + u));
            if (m < inf) {
                const int k = atomicAdd(&ne, 1);
                eu[k] = u;
                em[k] = m;
            }
        }
    }
    __syncthreads();
    const int m = ne, vv = blockIdx.x * 256 + tid;
    if (m == 0 || vv >= nv) return;
    double best = inf;
#pragma unroll 4
    for (int k = 0; k < m; ++k) best = fmin(best, __dadd_rn(em[k], __ldg(ds.vtab + (size_t)eu[k] * nv + vv)));
    if (best < inf) atomicMin((unsigned long long *)(ds.warm_est + vv), (unsigned long long)__double_as_longlong(best));
}

// Each obstacle vertex's tree parent: the in-neighbour u with the least
// estimate(u) + |u - v| (of equal values the smaller id), and that link's
// FP64 length as the fixpoint adds it. The in-edges are read where the edge
// lists take them from (the source columns of the vertex's bit row, then its
// kept obstacle-vertex list), so the lists can be built meanwhile. A group of
// kWarmGrp lanes per vertex, each over every kWarmGrp-th source and kept
// edge, then the lexicographic minimum across the group.
constexpr int kWarmGrp = 8;
__global__ void __launch_bounds__(256) k_warm_tree(const __grid_constant__ DevScene ds) {
    chain_start();
    const int t = blockIdx.x * 256 + threadIdx.x, vv = t / kWarmGrp, gl = t % kWarmGrp;
    const bool act = vv < ds.n_vert;  // every lane reaches the shuffles
    const int ns = ds.n_src;
    double best = __longlong_as_double(0x7ff0000000000000ll), blen = 0.0;
    int bp = -1;
    auto take = [&](int u, double len) {
        const double est = u < ns ? 0.0 : ds.warm_est[u - ns];
        const double c = __dadd_rn(est, len);
        if (est < kEstNone && (c < best || (c == best && u < bp))) {  // no estimate: u is not reached
            best = c;
            bp = u;
            blen = len;
        }
    };
    if (act) {
        const uint32_t *row = ds.vis_bits + (size_t)vv * ds.vis_words;
        for (int u = gl; u < ns; u += kWarmGrp)
            if ((row[u >> 5] >> (u & 31)) & 1u) take(u, edge_len(ds, u, ns + vv));
        for (int j = ds.st_start[vv] + gl, j1 = ds.st_start[vv + 1]; j < j1; j += kWarmGrp) take(ds.st_src[j], ds.st_len[j]);
    }
#pragma unroll
    for (int o = kWarmGrp / 2; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o), ol = __shfl_xor_sync(0xffffffffu, blen, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        if (ob < best || (ob == best && (unsigned)op < (unsigned)bp)) {
            best = ob;
            bp = op;
            blen = ol;
        }
    }
    if (act && gl == 0) {
        ds.warm_tpar[vv] = bp;
        ds.warm_tlen[vv] = blen;
    }
}

// Checks every obstacle vertex against the fixpoint's pull from the tree's
// state: the least (cost(u) + |u - v|, u) over its valid in-edges (u a
// source, or v inside u's shadow cone, from u's parent), with the arithmetic
// and the order of the fixpoint kernels' pulls. The vertices whose pull
// differs from their state are listed (ds.dirtyl[0], count in
// ds.counters[6]): they are the fixpoint's first round; every other vertex
// already satisfies its equation.
__global__ void __launch_bounds__(256) k_warm_verify(const __grid_constant__ DevScene ds) {
    chain_start();
    const int t = blockIdx.x * 256 + threadIdx.x, vv = t / kWarmGrp, gl = t % kWarmGrp;
    const bool act = vv < ds.n_vert;  // every lane reaches the shuffles
    const int ns = ds.n_src, v = ns + (act ? vv : 0);
    const int2 vl = ds.gen_lat[v];
    long long best = 0x7ff0000000000000ll;  // +inf bits
    int bpar = -1;
    const int e0 = act ? ds.in_start[vv] : 0, e1 = act ? ds.in_start[vv + 1] : 0;
    for (int e = e0 + gl; e < e1; e += kWarmGrp) {  // in generator order within the lane
        const int u = ds.in_src[e];
        const double cu = ds.warm_cost[u];
        const int pu = ds.warm_par[u];
        const int2 ul = ds.gen_lat[u];
        const int4 w4 = ds.gen_wedge[u];
        int dx = 0, dy = 0;
        if (pu >= 0) arrival_dir(ds, pu, ul, dx, dy);
        const short4 w = make_short4((short)w4.x, (short)w4.y, (short)w4.z, (short)w4.w);
        const bool valid = (__double_as_longlong(cu) < 0x7ff0000000000000ll) &
                           ((u < ns) | ((pu >= 0) & in_shadow_cone(dx, dy, w, vl.x - ul.x, vl.y - ul.y)));
        const long long cand = __double_as_longlong(__dadd_rn(cu, ds.in_len[e]));
        if (valid & (cand < best)) {
            best = cand;
            bpar = u;
        }
    }
#pragma unroll
    for (int o = kWarmGrp / 2; o > 0; o >>= 1) {  // the fixpoint's lexicographic minimum over the group
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, bpar, o);
        if (ob < best || (ob == best && (unsigned)op < (unsigned)bpar)) {
            best = ob;
            bpar = op;
        }
    }
    if (act && gl == 0 && (best != __double_as_longlong(ds.warm_cost[v]) || bpar != ds.warm_par[v]))
        ds.dirtyl[0][atomicAdd(ds.counters + 6, 1)] = v;
}

constexpr int kFoldThreads = 1024;
constexpr int kFoldPer = (kWarmMaxGen + kFoldThreads - 1) / kFoldThreads;  // generators per thread

// Shared memory of the tree fold for n generators.
__host__ __device__ __forceinline__ size_t fold_bytes(int n) {
    auto up = [](size_t x) { return (x + 15) & ~(size_t)15; };
    return 2 * up(8 * (size_t)n) + 3 * up(2 * (size_t)n) + up(4 * (size_t)n) + up(4 * ((size_t)n + 1));
}

// Costs along the tree, one CTA: the depth of every generator below its root
// by pointer doubling; the reached vertices sorted by depth; then one warp
// adds each level's links onto their parents' costs, level after level.
// Roots are the sources (cost 0) and vertices without a tree parent (not
// reached: +inf). A cycle of tree links (none is expected: estimates grow
// strictly along every link) would never reach a source, so its vertices
// are left unreached, as are the ones hanging from it.
__global__ void __launch_bounds__(kFoldThreads) k_warm_fold(const __grid_constant__ DevScene ds) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    chain_start();
    __shared__ long long wsum[32];
    __shared__ int s_maxd;
    const int n = ds.n_gen, ns = ds.n_src, tid = threadIdx.x, lane = tid & 31;
#ifdef SPM_COUNT
    long long tf[5];
    tf[0] = clock64();
#endif
    auto up = [](size_t x) { return (x + 15) & ~(size_t)15; };
    unsigned char *p = sm_raw;
    double *cost = (double *)p;             p += up(8 * (size_t)n);
    double *olen = (double *)p;             p += up(8 * (size_t)n);  // tree-link lengths, in `order`
    short *par = (short *)p;                p += up(2 * (size_t)n);
    unsigned *ad = (unsigned *)p;           p += 2 * up(2 * (size_t)n);  // root (low 16 bits) | depth (high 16)
    unsigned *order = (unsigned *)p;        p += up(4 * (size_t)n);  // by depth: vertex | parent << 16
    int *level = (int *)p;                  // n + 1: vertices per depth, then level ends
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    for (int g = tid; g < n; g += kFoldThreads) {
        const int pg = g < ns ? g : ds.warm_tpar[g - ns];
        par[g] = (short)pg;
        ad[g] = (unsigned)(pg < 0 ? g : pg) | (g < ns || pg < 0 ? 0u : 1u << 16);
        cost[g] = g < ns ? 0.0 : inf;
    }
    for (int d = tid; d <= n; d += kFoldThreads) level[d] = 0;
    if (tid == 0) s_maxd = 0;
    __syncthreads();
#ifdef SPM_COUNT
    tf[1] = clock64();
#endif
    // pointer doubling: each word becomes (the root, the links to it)
    for (int it = 0; it < 16; ++it) {
        unsigned was[kFoldPer], now[kFoldPer];
#pragma unroll
        for (int k = 0; k < kFoldPer; ++k) {
            const int g = tid + k * kFoldThreads;
            if (g < n) {
                const unsigned x = ad[g], y = ad[x & 0xffffu];
                was[k] = x;
                now[k] = (y & 0xffffu) | (min((x >> 16) + (y >> 16), 65535u) << 16);
            }
        }
        __syncthreads();
        int ch = 0;
#pragma unroll
        for (int k = 0; k < kFoldPer; ++k) {
            const int g = tid + k * kFoldThreads;
            if (g < n) {
                ch |= (now[k] ^ was[k]) & 0xffffu;
                ad[g] = now[k];
            }
        }
        if (!__syncthreads_or(ch)) break;
    }
#ifdef SPM_COUNT
    tf[2] = clock64();
#endif
    // a vertex is reached when its chain ends at a source (a chain caught in
    // a cycle never does); its depth is then at most n
    int md = 0;
    for (int g = ns + tid; g < n; g += kFoldThreads)
        if ((int)(ad[g] & 0xffffu) < ns) {
            const int d = (int)(ad[g] >> 16);
            atomicAdd(&level[d - 1], 1);
            md = max(md, d);
        }
    if (md) atomicMax(&s_maxd, md);
    __syncthreads();
    // exclusive scan of the level sizes, each thread a run of kFoldPer + 1 depths
    {
        constexpr int kRun = kFoldPer + 1;
        const int d0 = tid * kRun;
        long long mine = 0;
        for (int d = d0; d < d0 + kRun && d <= n; ++d) mine += level[d];
        long long run = cta_exclusive_scan(mine, wsum);
        for (int d = d0; d < d0 + kRun && d <= n; ++d) {
            const int c = level[d];
            level[d] = (int)run;
            run += c;
        }
    }
    __syncthreads();
    for (int g = ns + tid; g < n; g += kFoldThreads)
        if ((int)(ad[g] & 0xffffu) < ns) {  // level[k] ends as the end of depth k + 1
            const int i = atomicAdd(&level[(int)(ad[g] >> 16) - 1], 1);
            order[i] = (unsigned)g | ((unsigned)par[g] << 16);
            olen[i] = ds.warm_tlen[g - ns];
        }
    __syncthreads();
#ifdef SPM_COUNT
    tf[3] = clock64();
#endif
    if (tid < 32) {
        // one level after the other; a lane's first item of the next level
        // (vertex, parent, length) is loaded before this level's sums, so a
        // level costs one dependent load, one add and one store
        const int maxd = s_maxd;
        int lo = 0, hi = maxd > 0 ? level[0] : 0, nhi = maxd > 1 ? level[1] : hi;
        unsigned o = lane < hi ? order[lane] : 0u;
        double l = lane < hi ? olen[lane] : 0.0;
        for (int k = 0; k < maxd; ++k) {
            const double cp = cost[o >> 16];  // the one load on the chain, issued first
            const int ni = hi + lane, nnhi = k + 2 < maxd ? level[k + 2] : nhi;
            const unsigned no = ni < nhi ? order[ni] : 0u;
            const double nl = ni < nhi ? olen[ni] : 0.0;
            if (lo + lane < hi) cost[o & 0xffffu] = __dadd_rn(cp, l);
            for (int i = lo + 32 + lane; i < hi; i += 32) {  // levels wider than a warp
                const unsigned oi = order[i];
                cost[oi & 0xffffu] = __dadd_rn(cost[oi >> 16], olen[i]);
            }
            __syncwarp();
            lo = hi;
            hi = nhi;
            nhi = nnhi;
            o = no;
            l = nl;
        }
    }
    __syncthreads();
#ifdef SPM_COUNT
    tf[4] = clock64();
    if (tid == 0) {  // fold phases (SM cycles): loads, doubling, sort, level fold
        SPM_CNT(2, tf[1] - tf[0]);
        SPM_CNT(3, tf[2] - tf[1]);
        SPM_CNT(4, tf[3] - tf[2]);
        SPM_CNT(12, tf[4] - tf[3]);
    }
#endif
    for (int g = tid; g < n; g += kFoldThreads) {
        const bool ok = g < ns || (int)(ad[g] & 0xffffu) < ns;
        ds.warm_cost[g] = ok ? cost[g] : inf;
        ds.warm_par[g] = ok ? (int)par[g] : -1;
    }
}

// shared memory of the tree fold and of the table build, granted once per process
static bool fold_smem_ok() {
    static const bool ok = [] {
        if (cudaFuncSetAttribute(k_warm_fold, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fold_bytes(kWarmMaxGen)) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_vtab_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kVtabWarps * vtab_warp_bytes(kVtabMaxVert))) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    }();
    return ok;
}

bool vtab_possible(const DevScene &ds) {
    return ds.st_start && ds.st_len && ds.n_vert >= kVtabMinVert && ds.n_vert <= kVtabMaxVert &&
           ds.n_gen <= kWarmMaxGen && (ds.fix_launch & (kFixSoloSure | kFixClusterSure)) && fold_smem_ok();
}

// A compute with these fixpoint launches starts from the table's tree.
static bool warm_start_used(const DevScene &ds, int fix) {
    return ds.warm && ds.vtab && ds.n_vert > 0 && (fix & (kFixSoloSure | kFixClusterSure));
}

cudaError_t launch_vtab_build(const DevScene &ds, double *tab, int32_t *counter, cudaStream_t st) {
    if (!vtab_possible(ds)) return cudaErrorInvalidValue;
    const size_t smem = kVtabWarps * vtab_warp_bytes(ds.n_vert);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vtab_build, 32 * kVtabWarps, smem);
    const int need = (ds.n_vert + kVtabWarps - 1) / kVtabWarps;
    const int blocks = std::max(1, std::min(need, std::max(sms, 1) * std::max(per_sm, 1)));
    cudaMemsetAsync(counter, 0, 2 * sizeof(int32_t), st);  // [0] roots taken, [1] the most rounds a root took
    k_vtab_build<<<blocks, 32 * kVtabWarps, smem, st>>>(ds, tab, counter);
    return cudaGetLastError();
}

void launch_vertex_phase(const DevScene &ds, cudaStream_t st, const VertexSide *side) {
    int f = ds.fix_launch;
    if (g_many_cta_override.load() && !(f & kFixSoloSure)) f &= ~(kFixCluster | kFixClusterSure);  // test hook
    // the warm start needs a fixpoint kernel that takes it (the many-CTA one
    // always starts from the sources)
    const bool warm = warm_start_used(ds, f);
    // one kernel sets every per-compute start value (out-degrees, cursors,
    // the source columns of the bit matrix, counters, estimates)
    {
        DevScene arg = ds;
        arg.warm = warm ? 1 : 0;
        const long long items = std::max<long long>(
            ds.n_gen + 1, ds.st_start ? (long long)ds.n_vert * ((ds.n_src + 31) / 32) : 0);
        k_vertex_prep<<<(int)std::max(1LL, std::min((items + 255) / 256, 152LL * 4)), 256, 0, st>>>(arg);
    }
    if (ds.n_vert > 0) {
        const size_t bytes = sizeof(uint32_t) * (size_t)ds.n_vert * ds.vis_words;
        // the obstacle-vertex pairs come from the scene's static bits; the
        // pair kernel then tests the source columns only (with kept edge
        // lists only they are read: the prep kernel cleared them)
        if (!ds.st_start) {
            if (ds.vis_static) cudaMemcpyAsync(ds.vis_bits, ds.vis_static, bytes, cudaMemcpyDeviceToDevice, st);
            else cudaMemsetAsync(ds.vis_bits, 0, bytes, st);
        }
        launch_pairs(ds, st, false);
        const int eb = (ds.n_vert + 7) / 8;  // one warp per row
        if (warm && side) {
            // the tree's estimates, parents and fold read the source columns
            // and kept lists themselves: the edge lists, which only the
            // verification and the fixpoint read, are built beside them
            cudaEventRecord(side->fork, st);
            cudaStreamWaitEvent(side->st, side->fork, 0);
            k_edges_count<<<eb, 256, 0, side->st>>>(ds);
            launch_chained(k_edges_scan, dim3(1), dim3(1024), 0, side->st, ds);
            launch_chained(k_edges_fill, dim3(eb), dim3(256), 0, side->st, ds);
            cudaEventRecord(side->join, side->st);
        } else {
            launch_chained(k_edges_count, dim3(eb), dim3(256), 0, st, ds);
            launch_chained(k_edges_scan, dim3(1), dim3(1024), 0, st, ds);
            launch_chained(k_edges_fill, dim3(eb), dim3(256), 0, st, ds);
        }
    } else {
        cudaMemsetAsync(ds.in_start, 0, sizeof(int32_t) * (ds.n_vert + 1), st);
    }
    DevScene arg = ds;
    int max_rounds = fixpoint_round_cap(ds.n_gen);
    void *args[] = {&arg, &max_rounds};
    // each fixpoint kernel checks on the device whether the graph is its
    // own; the scene's bounds on the edge count skip the launches that
    // cannot apply
    arg.warm = warm ? 1 : 0;
    if (arg.warm) {
        const int vb = (ds.n_vert + 255) / 256;
        launch_chained(k_warm_entry, dim3(vb, (ds.n_vert + kEntryRows - 1) / kEntryRows), dim3(256), 0, st, arg);
        const int gb = (ds.n_vert * kWarmGrp + 255) / 256;
        launch_chained(k_warm_tree, dim3(gb), dim3(256), 0, st, arg);
        launch_chained(k_warm_fold, dim3(1), dim3(kFoldThreads), fold_bytes(ds.n_gen), st, arg);
        if (side && ds.n_vert > 0) {  // the edge lists are complete before the verification reads them
            cudaStreamWaitEvent(st, side->join, 0);
            k_warm_verify<<<gb, 256, 0, st>>>(arg);
        } else {
            launch_chained(k_warm_verify, dim3(gb), dim3(256), 0, st, arg);
        }
    }
    if (f & kFixSolo) launch_chained(k_sssp_solo, dim3(1), dim3(kSoloThreads), (size_t)ds.solo_smem, st, arg, max_rounds);
    if (f & kFixCluster) {
        if (f & kFixClusterWide)
            launch_chained(k_sssp_cluster<kClCtasWide>, dim3(kClCtasWide), dim3(kClThreads), (size_t)kClSmem, st, arg,
                           max_rounds);
        else
            launch_chained(k_sssp_cluster<kClCtas>, dim3(kClCtas), dim3(kClThreads), (size_t)kClSmem, st, arg, max_rounds);
    }
    if (!(f & (kFixSoloSure | kFixClusterSure))) {
        cudaLaunchCooperativeKernel((const void *)k_sssp, dim3(ds.sssp_blocks), dim3(kSsspThreads), args, 0, st);
        k_finalize<<<(ds.n_gen + 255) / 256, 256, 0, st>>>(ds);
    }
}

int solo_smem_bytes() {
    return cudaFuncSetAttribute(k_sssp_solo, cudaFuncAttributeMaxDynamicSharedMemorySize, kSoloSmem) == cudaSuccess
               ? kSoloSmem
               : (cudaGetLastError(), 0);
}

int sssp_grid_blocks() {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sssp, kSsspThreads, 0);
    per_sm = per_sm < 1 ? 1 : (per_sm > 2 ? 2 : per_sm);
    return (sms > 0 ? sms : 1) * per_sm;
}

int count_kernel_launches_vertex() { return 6; }

int vis_resident_blocks() {
    static int blocks = 0;
    if (!blocks) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vis_pairs, kVisThreads, 0);
        blocks = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    }
    return blocks;
}

void launch_vert_maps(const DevScene &ds, cudaStream_t st, float *maps) {
    if (ds.n_vert > 0) k_vert_maps<<<(ds.n_vert + 7) / 8, 256, 0, st>>>(ds, maps);
}

int sssp_batched_grid_blocks() {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sssp_b, kSsspThreads, 0);
    per_sm = per_sm < 1 ? 1 : (per_sm > 2 ? 2 : per_sm);
    return (sms > 0 ? sms : 1) * per_sm;
}

void launch_vertex_phase_batched(const BatchDev &b, cudaStream_t st) {
    k_prepare_b<<<152 * 4, 256, 0, st>>>(b);
    k_vis_pairs_b<<<vis_resident_blocks(), kVisThreads, 0, st>>>(b);
    k_edges_count_b<<<152 * 4, 256, 0, st>>>(b);
    k_edges_scan_b<<<b.n, 1024, 0, st>>>(b);
    k_edges_fill_b<<<152 * 4, 256, 0, st>>>(b);
    BatchDev arg = b;
    void *args[] = {&arg};
    if (b.cl_grid > 0) {  // the clusters first; the many-CTA kernel takes what they leave
        cudaMemsetAsync(b.cl_counter, 0, sizeof(int32_t), st);
        k_sssp_cluster_b<<<b.cl_grid, kClThreads, kClSmem, st>>>(b);
    } else {
        cudaMemsetAsync(b.cl_done, 0, sizeof(int32_t) * b.n, st);
    }
    if (!b.cl_all)
        cudaLaunchCooperativeKernel((const void *)k_sssp_b, dim3(b.sssp_blocks), dim3(kSsspThreads), args, 0, st);
    k_finalize_b<<<152 * 4, 256, 0, st>>>(b);
}

int cluster_batched_grid() {
    if (!cluster_smem_ok() || g_many_cta_override.load()) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClCtas);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = kClSmem;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_sssp_cluster_b, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return clusters * kClCtas;  // resident clusters only: they take scenes from a counter
}

}  // namespace spm

extern "C" void spm_debug_set_round_cap(int32_t n) { spm::g_round_cap_override.store(n > 0 ? n : 0); }
extern "C" void spm_debug_set_many_cta_fixpoint(int32_t on) { spm::g_many_cta_override.store(on ? 1 : 0); }

#ifdef SPM_COUNT
// Instrumentation build only: reads and clears this unit's work counters.
extern "C" int spm_debug_counters_vertex(unsigned long long *out32) {
    cudaDeviceSynchronize();
    if (cudaMemcpyFromSymbol(out32, spm::g_count, sizeof(unsigned long long) * 32) != cudaSuccess) return 1;
    unsigned long long z[32] = {0};
    cudaMemcpyToSymbol(spm::g_count, z, sizeof z);
    return 0;
}
#endif
