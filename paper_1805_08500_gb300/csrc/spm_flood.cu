// spm_flood.cu -- per-tile candidate lists by flooding each generator's
// potentially visible tiles (the per-tile culling step of the pixel pass).
//
// For a point generator g (point source, segment endpoint, obstacle vertex),
// the pixels that see g and lie in its shadow cone form a region that is
// star-shaped from g: the segment from g to any such pixel stays inside the
// cone and sees g all along. Every tile that segment crosses therefore holds
// visible points. A breadth-first flood over tiles from g's tile, expanding a
// tile only when it meets the cone and is not provably hidden from g (by the
// angular depth map below), thus reaches every tile where g can win (tiles
// are closed rectangles that tile the plane; 8-neighbour steps follow any
// segment). Each reached tile gets g in its candidate list. One CTA floods one
// generator, a breadth-first level at a time. Segment interiors, points
// outside the tile grid and floods whose level outgrows the frontier go to a
// global list that every tile scans. Any failure of the lists (pair capacity)
// sets a flag and the pixel pass falls back to scanning every generator.
#include <cuda_runtime.h>

#include <algorithm>

#include "spm_device.cuh"
#include "spm_internal.h"

namespace spm {
namespace {

constexpr int kFloodThreads = 256;  // one CTA floods one generator at a time
constexpr int kFront = 1024;        // frontier tiles per breadth-first level
constexpr int kFloodPolyBits = 65536;  // polygons tracked for insertion (beyond: inserted again, harmless)

// Full area of tile (tx, ty) in lattice units: closed rectangle, neighbours
// share edges. Pixel i covers [i * pitch, (i + 1) * pitch].
__device__ __forceinline__ int4 tile_area(const DevScene &ds, int tx, int ty) {
    const int px = ds.S * ds.Wx / ds.Nx, py = ds.S * ds.Wy / ds.Ny;
    const int T = ds.tile;
    return make_int4(tx * T * px, ty * T * py, min((tx + 1) * T, ds.Nx) * px, min((ty + 1) * T, ds.Ny) * py);
}

__device__ __forceinline__ bool cone_meets_box(int ct, int4 c, int2 v, int4 box) {
    if (ct == kConeNone) return true;
    if (ct == kConeEmpty) return false;
    const int cx[4] = {box.x, box.z, box.x, box.z}, cy[4] = {box.y, box.y, box.w, box.w};
    bool out1 = true, out2 = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int wx = cx[k] - v.x, wy = cy[k] - v.y;
        out1 &= cross32(c.x, c.y, wx, wy) < 0;
        out2 &= cross32(wx, wy, c.z, c.w) < 0;
    }
    return !(out1 || out2);
}

__device__ __forceinline__ void push_global(const DevScene &ds, int g) {
    ds.glob_list[atomicAdd(&ds.flood_counts[1], 1)] = g;
}

// Angular depth map of one generator g (shadow volumes, in the spirit of the
// shadow construction of Sec. 3.1): directions around g are cut into kAng
// bins of a pseudo-angle; depth2[b] is an upper bound on the squared distance
// from g at which every ray of bin b has crossed a front-facing obstacle edge
// (g strictly on its outer side), i.e. entered an obstacle interior. A tile is
// hidden from g when every bin its corners span has depth2 at most the tile's
// squared nearest distance: each of its points lies beyond an obstacle
// interior on its ray. Along an edge's line the crossing distance is convex in
// the ray angle, so over a bin it peaks at one of the two boundary rays; the
// boundary directions are exact multiples of 1/512, which makes the dot
// products exact in integers and leaves a few float roundings (covered by a
// 1e-5 relative margin). Polygons enter the map as the flood reaches their
// tiles, so every test is conservative; unions of polygons (walls that
// overlap at posts) hide tiles that no single polygon hides.
constexpr int kAng = kAngBins;      // pseudo-angle bins over [0, 4)
constexpr int kAngQ = kAng / 4;     // bins per quadrant (boundary m is pseudo-angle m / kAngQ)
constexpr int kInsCap = 1024;       // polygons inserted per level

// Pseudo-angle difference b - a wrapped into (-2, 2].
__device__ __forceinline__ float pang_diff(float a, float b) {
    float d = b - a;
    if (d > 2.f) d -= 4.f;
    if (d <= -2.f) d += 4.f;
    return d;
}

// Direction of bin boundary m, scaled by kAngQ: integer components.
__device__ __forceinline__ int2 boundary_dir(int m) {
    const int mm = m & (kAng - 1), f = mm & (kAngQ - 1);
    switch (mm / kAngQ) {
        case 0: return make_int2(kAngQ - f, f);
        case 1: return make_int2(-f, kAngQ - f);
        case 2: return make_int2(-(kAngQ - f), -f);
        default: return make_int2(f, -(kAngQ - f));
    }
}

struct FloodSmem {
    float depth2[kAng];
    int front[2][kFront];  // current / next breadth-first level
    int flag[kFront];      // 0 visible, 1 hidden, 2 outside the cone
    int ins[kInsCap];      // polygons to insert before this level's tests
    int cnt[2];
    int n_ins;
    int overflow;
    int ins_dropped;       // a polygon was left out of the map (insertion list full)
};

// Is the closed box hidden from g (lattice point, not inside the box) by the
// depth map? A group of G lanes (lane gl of mask gmask) tests G of the
// spanned bins at a time (a tile near g spans hundreds of bins, a far one a
// few).
template <int G>
__device__ bool box_hidden_ang(const float *depth2, int2 g, int4 box, int gl, unsigned gmask, int stride) {
    const long long dx = max(max(box.x - g.x, g.x - box.z), 0), dy = max(max(box.y - g.y, g.y - box.w), 0);
    const float mind2 = (float)(dx * dx + dy * dy) * (1.f - 1e-6f);
    const float c0 = pang(0.5f * (float)(box.x + box.z) - (float)g.x, 0.5f * (float)(box.y + box.w) - (float)g.y);
    float lo = 0.f, hi = 0.f;
    const int cx[4] = {box.x, box.z, box.x, box.z}, cy[4] = {box.y, box.y, box.w, box.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float d = pang_diff(c0, pang((float)(cx[k] - g.x), (float)(cy[k] - g.y)));
        lo = fminf(lo, d);
        hi = fmaxf(hi, d);
    }
    const int k0 = (int)floorf((c0 + lo - kAngEps) / kAngW), k1 = (int)floorf((c0 + hi + kAngEps) / kAngW);
    for (int k = k0; k <= k1; k += G) {
        const int kk = k + gl;
        const bool h = kk > k1 || depth2[stride * ((kk + 2 * kAng) & (kAng - 1))] <= mind2;
        if (!__all_sync(gmask, h)) return false;
    }
    return true;
}
__device__ __forceinline__ bool box_hidden_ang_warp(const float *depth2, int2 g, int4 box, int lane, int stride = 1) {
    return box_hidden_ang<32>(depth2, g, box, lane, 0xffffffffu, stride);
}

// One warp inserts polygon q's front-facing edges into the depth map, the
// lanes spread over each edge's bins.
template <bool MAPS>
__device__ void insert_polygon_warp(const DevScene &ds, float *depth2, float *lo2, int2 g, int q, int lane,
                                    float plen, int stride = 1) {
    const int b = ds.poly_off[q], m = ds.poly_off[q + 1] - b;
    const int2 mine = lane < m ? ds.poly_v[b + lane] : make_int2(0, 0);  // vertex `lane`, one load per lane
    for (int i = 0; i < m; ++i) {
        const int in = i + 1 == m ? 0 : i + 1;
        const int2 a = make_int2(__shfl_sync(0xffffffffu, mine.x, i), __shfl_sync(0xffffffffu, mine.y, i));
        const int2 c = make_int2(__shfl_sync(0xffffffffu, mine.x, in), __shfl_sync(0xffffffffu, mine.y, in));
        if (orient32(a.x, a.y, c.x, c.y, g.x, g.y) >= 0) continue;  // not front-facing
        // line normal n (left of a -> c); g is on its negative side, so
        // n . (a - g) > 0 and n . u > 0 for every ray u that meets the edge
        const int nx = -(c.y - a.y), ny = c.x - a.x;
        const long long N = (long long)nx * (a.x - g.x) + (long long)ny * (a.y - g.y);
        const float fN2 = (float)N * (float)N;
        // no ray crosses the line closer than its distance from g
        const float h2 = __fdividef(fN2, (float)nx * (float)nx + (float)ny * (float)ny) * (1.f - 1e-5f);
        // the edge runs clockwise seen from g: its angle range goes
        // counter-clockwise from c to a
        const float lo = pang((float)(c.x - g.x), (float)(c.y - g.y));
        const float hi = lo + fmodf(pang((float)(a.x - g.x), (float)(a.y - g.y)) - lo + 4.f, 4.f);
        const int k0 = (int)ceilf((lo + kAngEps) / kAngW), k1 = (int)floorf((hi - kAngEps) / kAngW) - 1;
        auto bdist2 = [&](int mb) {  // squared crossing distance along boundary ray mb, rounded up
            const int2 u = boundary_dir(mb);
            const float fD = (float)(nx * u.x + ny * u.y);  // exact: |n| < 2^16, |u| <= 512
            return __fdividef(fN2 * (float)(u.x * u.x + u.y * u.y), fD * fD) * (1.f + 1e-5f);
        };
        for (int k = k0 + lane; k <= k1; k += 32) {
            int *slot = (int *)&depth2[stride * (k & (kAng - 1))];
            if (__int_as_float(*slot) <= h2) continue;  // this edge cannot lower the bin
            atomicMin(slot, __float_as_int(fmaxf(bdist2(k), bdist2(k + 1))));  // non-negative floats order as ints
        }
        // Lower bound: a ray entering an obstacle crosses a front-facing edge
        // (or passes a vertex of one) at a point of some piece of it, no
        // nearer than that piece's distance from g. Pieces of at most plen
        // lattice units; every bin touching a piece's closed angle range.
        if (!MAPS) continue;
        const float ax = (float)(a.x - g.x), ay = (float)(a.y - g.y), ex = (float)(c.x - a.x), ey = (float)(c.y - a.y);
        const float el = sqrtf(ex * ex + ey * ey);
        const int np = max(1, (int)ceilf(el / plen));
        for (int j = lane; j < np; j += 32) {
            const float t0 = (float)j / (float)np, t1 = j + 1 == np ? 1.f : (float)(j + 1) / (float)np;
            const float px0 = ax + t0 * ex, py0 = ay + t0 * ey, px1 = ax + t1 * ex, py1 = ay + t1 * ey;
            const float dx = px1 - px0, dy = py1 - py0, dd = dx * dx + dy * dy;
            const float tt = dd > 0.f ? fminf(fmaxf(-(px0 * dx + py0 * dy) / dd, 0.f), 1.f) : 0.f;
            const float cx = px0 + tt * dx, cy = py0 + tt * dy;
            const float d2 = fmaxf((cx * cx + cy * cy) * (1.f - 2e-5f) - 0.05f, 0.f);
            const float plo = pang(px1, py1), phi = plo + fmodf(pang(px0, py0) - plo + 4.f, 4.f);
            const int b0 = (int)floorf((plo - kAngEps) / kAngW), b1 = (int)floorf((phi + kAngEps) / kAngW);
            for (int k = b0; k <= b1; ++k)
                atomicMin((int *)&lo2[stride * ((k + 2 * kAng) & (kAng - 1))], __float_as_int(d2));
        }
    }
}

// Floods generator g of scene ds: one CTA, a breadth-first level at a time.
// MAPS: also keep g's depth map (with the lower-bound bins) for the pixel pass.
template <bool MAPS>
__device__ void flood_one(const DevScene &ds, FloodSmem &sm, unsigned *fdyn, int g) {
    const int tid = threadIdx.x;
    const int ntiles = ds.tiles_x * ds.tiles_y, words = (ntiles + 31) / 32;
    const int pwords = ds.n_poly <= kFloodPolyBits ? (ds.n_poly + 31) / 32 : 0;
    unsigned *visited = fdyn, *seen = fdyn + words;  // tiles reached; polygons inserted
    // with maps: lower bound of the squared distance at which a ray of each
    // bin can first meet an obstacle (after the bitmaps in dynamic smem)
    float *lo2 = reinterpret_cast<float *>(fdyn + words + pwords);
    const int tpx = ds.tile * (ds.S * ds.Wx / ds.Nx), tpy = ds.tile * (ds.S * ds.Wy / ds.Ny);
    // mode 3 floods from geometry alone (every generator, no cone): it runs
    // before the vertex costs exist, and the pixel pass applies cost and cone
    const bool geometric = ds.flood_mode == 3;
    const float plen = fmaxf(1.f, 0.125f * (float)min(tpx, tpy));  // lower-bound piece length
    constexpr bool maps = MAPS;
    if (ds.gen_map_ok && tid == 0) ds.gen_map_ok[g] = 0;  // set again when the map is complete
    SPM_T0();
    if (!geometric && !(ds.gen_costf[g] < INFINITY)) return;
    const int kind = ds.gen_kind[g];
    const int ct = kind == kVert && !geometric ? ds.gen_ctype[g] : kConeNone;
    if (ct == kConeEmpty) return;
    if (kind == kSegI) {
        if (tid == 0) push_global(ds, g);
        return;
    }
    const int2 gl = ds.gen_lat[g];
    const int4 cone = ct != kConeNone ? ds.gen_cone[g] : make_int4(0, 0, 0, 0);
    const int tx = gl.x >= 0 ? gl.x / tpx : -1, ty = gl.y >= 0 ? gl.y / tpy : -1;
    __syncthreads();  // the previous generator is done with smem
    for (int w = tid; w < words + pwords; w += kFloodThreads) fdyn[w] = 0u;
    for (int k = tid; k < kAng; k += kFloodThreads) sm.depth2[k] = INFINITY;
    if (maps)
        for (int k = tid; k < kAng; k += kFloodThreads) lo2[k] = INFINITY;
    if (tid == 0) {
        sm.cnt[0] = 0;
        sm.overflow = 0;
        sm.n_ins = 0;
        sm.ins_dropped = 0;
    }
    __syncthreads();
    // seeds: every tile whose closed area contains g (up to 4 when g lies on tile edges)
    if (tid < 4) {
        const int sx = tx - (tid & 1), sy = ty - ((tid >> 1) & 1);
        if (tx >= 0 && ty >= 0 && sx >= 0 && sy >= 0 && sx < ds.tiles_x && sy < ds.tiles_y) {
            const int4 a4 = tile_area(ds, sx, sy);
            if (gl.x >= a4.x && gl.x <= a4.z && gl.y >= a4.y && gl.y <= a4.w) {
                const int t0 = sy * ds.tiles_x + sx;
                if (!(atomicOr(&visited[t0 >> 5], 1u << (t0 & 31)) & (1u << (t0 & 31))))
                    sm.front[0][atomicAdd(&sm.cnt[0], 1)] = t0;
            }
        }
    }
    __syncthreads();
    SPM_LAP(0);
    if (sm.cnt[0] == 0) {  // g outside every tile: scanned by all tiles instead
        if (tid == 0) push_global(ds, g);
        return;
    }
#ifdef SPM_COUNT
    int n_tests = 0, n_levels = 0;
#endif
    int p = 0;
    for (;;) {
        if (sm.overflow) {  // a level outgrew the frontier: every tile scans g instead
            if (tid == 0) {
                push_global(ds, g);
                SPM_CNT(13, 1);
            }
            break;
        }
        const int nc = min(sm.cnt[p], kFront);
        if (nc == 0) break;
        const int *cur = sm.front[p];
        // A: the polygons in the frontier tiles' bins enter the depth map
        for (int q = tid; q < nc * 16; q += kFloodThreads) {  // (tile, one of its first 16 bins)
            const int i = q >> 4, j = q & 15;
            const int t = cur[i];
            const int4 area = tile_area(ds, t % ds.tiles_x, t / ds.tiles_x);
            const int bx0 = max(0, (area.x - ds.bin_x0) / ds.bin_size), by0 = max(0, (area.y - ds.bin_y0) / ds.bin_size);
            const int bx1 = min(ds.bin_nx - 1, (area.z - ds.bin_x0) / ds.bin_size);
            const int by1 = min(ds.bin_ny - 1, (area.w - ds.bin_y0) / ds.bin_size);
            const int nbx = bx1 - bx0 + 1, nby = by1 - by0 + 1;
            for (int jj = j; jj < nbx * nby; jj += 16) {
                const int bin = (by0 + jj / nbx) * ds.bin_nx + bx0 + jj % nbx;
                const int e = __ldg(ds.bin_start + bin + 1);
                for (int it = __ldg(ds.bin_start + bin); it < e; ++it) {
                    const int poly = __ldg(reinterpret_cast<const int *>(ds.bin_recs + it) + 4);
                    if (pwords) {
                        const unsigned bit = 1u << (poly & 31);
                        if (atomicOr(&seen[poly >> 5], bit) & bit) continue;
                    }
                    const int slot = atomicAdd(&sm.n_ins, 1);
                    if (slot < kInsCap) sm.ins[slot] = poly;  // beyond the cap: left out of the map
                    else sm.ins_dropped = 1;
                }
            }
        }
        __syncthreads();
        SPM_LAP(1);
        const int ni = min(sm.n_ins, kInsCap);
        for (int q = tid >> 5; q < ni; q += kFloodThreads / 32)
            insert_polygon_warp<MAPS>(ds, sm.depth2, lo2, gl, sm.ins[q], tid & 31, plen);
        __syncthreads();
        SPM_LAP(2);
#ifdef SPM_TIME
        spm_acc_[6] += 1;   // levels
        spm_acc_[7] += ni;  // polygons inserted
#endif
        // B: cone and depth-map test per frontier tile, a warp per tile
        for (int i = tid >> 5; i < nc; i += kFloodThreads / 32) {
            const int t = cur[i];
            const int4 area = tile_area(ds, t % ds.tiles_x, t / ds.tiles_x);
            int f = 2;
            if (cone_meets_box(ct, cone, gl, area)) {
                const bool inside = gl.x >= area.x && gl.x <= area.z && gl.y >= area.y && gl.y <= area.w;
                f = !inside && box_hidden_ang_warp(sm.depth2, gl, area, tid & 31) ? 1 : 0;
            }
            if ((tid & 31) == 0) sm.flag[i] = f;
        }
        if (tid == 0) {
            sm.cnt[p ^ 1] = 0;
            sm.n_ins = 0;
        }
        __syncthreads();
        SPM_LAP(3);
        // C: emit visible tiles, queue their fresh 8-neighbours
        int *nxt = sm.front[p ^ 1];
        for (int q = tid; q < nc * 9; q += kFloodThreads) {
            const int i = q / 9, k = q - 9 * i;
            const int f = sm.flag[i];
#ifdef SPM_COUNT
            if (k == 4 && f != 2) {
                SPM_CNT(11, 1);
                SPM_CNT(12, f == 0 ? 1 : 0);
            }
#endif
            if (f) continue;
            const int t = cur[i];
            if (k == 4) {
                const int slot = atomicAdd(&ds.flood_counts[0], 1);
                if (slot < ds.pair_cap) {
                    ds.pairs[slot] = make_int2(t, g);
                    atomicAdd(&ds.tile_count[t], 1);
                } else {
                    atomicOr(&ds.flood_counts[2], 1);
                }
                continue;
            }
            const int nx = t % ds.tiles_x + k % 3 - 1, ny = t / ds.tiles_x + k / 3 - 1;
            if (nx < 0 || ny < 0 || nx >= ds.tiles_x || ny >= ds.tiles_y) continue;
            const int nt = ny * ds.tiles_x + nx;
            if (atomicOr(&visited[nt >> 5], 1u << (nt & 31)) & (1u << (nt & 31))) continue;
            const int slot = atomicAdd(&sm.cnt[p ^ 1], 1);
            if (slot < kFront) nxt[slot] = nt;
            else sm.overflow = 1;
        }
#ifdef SPM_COUNT
        if (tid == 0) {
            ++n_levels;
            for (int i = 0; i < nc; ++i) n_tests += sm.flag[i] != 2;
        }
#endif
        __syncthreads();
        SPM_LAP(4);
        p ^= 1;
    }
#ifdef SPM_COUNT
    if (tid == 0) {
        SPM_CNT_MAX(14, n_tests);
        SPM_CNT_MAX(15, n_levels);
    }
#endif
    // keep the depth map for the pixel pass when it holds every polygon of
    // the reached tiles (no frontier overflow, nothing left out)
    if (maps && !sm.overflow && !sm.ins_dropped) {
        float2 *mp = ds.gen_maps + (size_t)g * kAng;
        for (int k = tid; k < kAng; k += kFloodThreads) mp[k] = make_float2(sm.depth2[k], lo2[k]);
        if (tid == 0) ds.gen_map_ok[g] = 1;
    }
    SPM_LAP(5);
    SPM_TFLUSH();
}

// Direct culling of the sources (generators [0, n_src)) in the geometric
// mode: few generators, each reaching much of the grid, which one CTA per
// generator would walk a breadth-first level at a time. Instead every
// polygon enters each source's depth map at once (a warp per (source,
// polygon), atomics into the source's map in global memory), and then every
// tile is tested against the complete map at once (a warp per (source,
// tile)). A tile that the map does not hide gets the source in its list.
// That is a superset of what the walk reaches -- the walk also stops at
// tiles cut off by hidden ones -- and every tile where the source can win is
// still in it: the map only hides points that lie beyond an obstacle
// interior on their ray. With every polygon in it the map is complete, and
// the pixel pass may use it.
__device__ __forceinline__ bool src_on_grid(const DevScene &ds, int g) {
    const int2 gl = ds.gen_lat[g];
    const int px = ds.S * ds.Wx / ds.Nx, py = ds.S * ds.Wy / ds.Ny;
    return ds.gen_kind[g] != kSegI && gl.x >= 0 && gl.y >= 0 && gl.x <= ds.Nx * px && gl.y <= ds.Ny * py;
}

// Before the sources' culling: empty maps and lists, the global list after
// the obstacle vertices' entries, the overflow flag as their flood left it.
__device__ __forceinline__ void src_prep(const DevScene &ds, int i0, int stride, bool counts) {
    const int nmap = ds.n_src * kAng, ntiles = ds.tiles_x * ds.tiles_y;
    for (int i = i0; i < max(nmap, ntiles); i += stride) {
        if (i < nmap) ds.gen_maps[i] = make_float2(INFINITY, INFINITY);
        if (i < ntiles) ds.tile_count[i] = 0;
        if (i < ds.n_src) ds.gen_map_ok[i] = 0;
    }
    if (counts && i0 < 4) ds.flood_counts[i0] = i0 == 1 || i0 == 2 ? ds.static_counts[i0] : 0;
}

template <bool MAPS>
__device__ __forceinline__ void src_insert(const DevScene &ds, int g, int q, int lane) {
    if (!src_on_grid(ds, g)) return;
    const int tpx = ds.tile * (ds.S * ds.Wx / ds.Nx), tpy = ds.tile * (ds.S * ds.Wy / ds.Ny);
    const float plen = fmaxf(1.f, 0.125f * (float)min(tpx, tpy));  // as in the flood
    float *mp = reinterpret_cast<float *>(ds.gen_maps + (size_t)g * kAng);
    insert_polygon_warp<MAPS>(ds, mp, mp + 1, ds.gen_lat[g], q, lane, plen, 2);
}

constexpr int kSrcGrp = 8;  // lanes per (source, tile) test: most tiles span few bins
template <bool MAPS>
__device__ __forceinline__ void src_tile(const DevScene &ds, int g, int t, int lane, unsigned gmask) {
    if (!src_on_grid(ds, g)) {  // segment interiors and sources off the grid: every tile scans them
        if (t == 0 && lane == 0) push_global(ds, g);
        return;
    }
    const int2 gl = ds.gen_lat[g];
    const int4 area = tile_area(ds, t % ds.tiles_x, t / ds.tiles_x);
    const bool inside = gl.x >= area.x && gl.x <= area.z && gl.y >= area.y && gl.y <= area.w;
    const float *mp = reinterpret_cast<const float *>(ds.gen_maps + (size_t)g * kAng);
    if (MAPS && t == 0 && lane == 0) ds.gen_map_ok[g] = 1;  // complete: the pixel pass may read it
    if (!inside && box_hidden_ang<kSrcGrp>(mp, gl, area, lane, gmask, 2)) return;
    if (lane == 0) {
        const int slot = atomicAdd(&ds.flood_counts[0], 1);
        if (slot < ds.pair_cap) {
            ds.pairs[slot] = make_int2(t, g);
            atomicAdd(&ds.tile_count[t], 1);
        } else {
            atomicOr(&ds.flood_counts[2], 1);
        }
    }
}

__global__ void k_src_prep(DevScene ds) {
    src_prep(ds, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, true);
}

template <bool MAPS>
__global__ void k_src_insert(DevScene ds) {
    const long long n = (long long)ds.n_src * ds.n_poly;
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w < n;
         w += (gridDim.x * (long long)blockDim.x) >> 5)
        src_insert<MAPS>(ds, (int)(w / ds.n_poly), (int)(w % ds.n_poly), threadIdx.x & 31);
}

// group of kSrcGrp lanes of the calling thread's warp
__device__ __forceinline__ unsigned src_group_mask() {
    return ((1u << kSrcGrp) - 1u) << ((threadIdx.x & 31) & ~(kSrcGrp - 1));
}

template <bool MAPS>
__global__ void k_src_tiles(DevScene ds) {
    const int ntiles = ds.tiles_x * ds.tiles_y;
    const long long n = (long long)ds.n_src * ntiles;
    const unsigned gmask = src_group_mask();
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / kSrcGrp; w < n;
         w += (gridDim.x * (long long)blockDim.x) / kSrcGrp)
        src_tile<MAPS>(ds, (int)(w / ntiles), (int)(w % ntiles), threadIdx.x % kSrcGrp, gmask);
}

// Automatic mode: flood only sparse visibility graphs (mazes); a dense one
// marks the lists unavailable and every tile scans every generator.
__device__ __forceinline__ bool flood_declined(const DevScene &ds) {
    if (ds.flood_mode != 0) return false;
    const double pairs = (double)ds.n_gen * (double)max(ds.n_vert, 1);
    return (double)ds.in_start[ds.n_vert] > 0.01 * pairs;
}

// Resident CTAs take generators from a work counter (flood_counts[3]) as
// they finish: flood depths vary widely, so a fixed stride would leave the
// kernel waiting for the CTAs that drew several deep generators.
// Generators [g0, g1) are flooded.
template <bool MAPS>
__global__ void __launch_bounds__(kFloodThreads, MAPS ? 6 : 8) k_flood(DevScene ds, int g0, int g1) {
    extern __shared__ unsigned fdyn[];
    __shared__ FloodSmem sm;
    __shared__ int next_g;
    if (flood_declined(ds)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ds.flood_counts[2] = 1;
        return;
    }
    for (;;) {
        if (threadIdx.x == 0) next_g = g0 + atomicAdd(&ds.flood_counts[3], 1);
        __syncthreads();
        const int g = next_g;
        __syncthreads();  // next_g is rewritten for the next generator
        if (g >= g1) break;
        flood_one<MAPS>(ds, sm, fdyn, g);
    }
}

// After the obstacle vertices' flood (keep = 1) its counts are saved; before
// the sources' flood (keep = 0) the lists start empty, the global list after
// the vertices' entries, the overflow flag as the vertices' flood left it,
// and the work counter from zero.
__global__ void k_flood_static(DevScene ds, int keep) {
    const int ntiles = ds.tiles_x * ds.tiles_y;
    if (!keep)
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) ds.tile_count[t] = 0;
    if (blockIdx.x == 0 && threadIdx.x < 4) {
        const int k = threadIdx.x;
        if (keep) {
            if (k < 3) ds.static_counts[k] = ds.flood_counts[k];
        } else {
            ds.flood_counts[k] = k == 1 || k == 2 ? ds.static_counts[k] : 0;
        }
    }
}



// Batched form: every (scene, generator) of the batch, one CTA each.
template <class T>
__device__ __forceinline__ int scene_of_b(const T *off, int n, T x) {
    int lo = 0, hi = n;  // last scene with off[s] <= x
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <bool ANY_MAPS>  // some scene of the batch keeps depth maps
__global__ void __launch_bounds__(kFloodThreads, ANY_MAPS ? 6 : 8) k_flood_b(const __grid_constant__ BatchDev b) {
    extern __shared__ unsigned fdyn[];
    __shared__ FloodSmem sm;
    const int total = b.flood_off[b.n];
    for (int i = blockIdx.x; i < total; i += gridDim.x) {  // (scene, generator) tasks: sources only when reusing
        const int sc = scene_of_b(b.flood_off, b.n, i);
        const DevScene &ds = b.scenes[sc];
        if (!ds.use_flood || ds.flood_mode == 2) continue;
        if (flood_declined(ds)) {
            if (threadIdx.x == 0) ds.flood_counts[2] = 1;
            continue;
        }
        if (ANY_MAPS && ds.use_maps && ds.gen_maps) flood_one<true>(ds, sm, fdyn, i - b.flood_off[sc]);
        else flood_one<false>(ds, sm, fdyn, i - b.flood_off[sc]);
    }
}

// Per-scene list state before a batched flood: counts zeroed, or the lists
// marked unavailable for scenes that scan; the depth maps of directly culled
// sources emptied.
__global__ void k_flood_reset_b(const __grid_constant__ BatchDev b) {
    const int total = b.tile_off[b.n];
    const long long nmap = b.src_map_off[b.n];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total + b.n + nmap;
         i += gridDim.x * (long long)blockDim.x) {
        if (i >= total + b.n) {
            const long long m = i - total - b.n;
            const int sc = scene_of_b(b.src_map_off, b.n, m);
            const DevScene &ds = b.scenes[sc];
            const long long e = m - b.src_map_off[sc];
            ds.gen_maps[e] = make_float2(INFINITY, INFINITY);
            if (e % kAng == 0) ds.gen_map_ok[e / kAng] = 0;
        } else if (i < total) {
            const int oi = scene_of_b(b.tile_off, b.n, (int32_t)i), sc = b.order[oi];
            b.scenes[sc].tile_count[i - b.tile_off[oi]] = 0;
        } else {  // reusing scenes: the global list after the vertices' entries
            const DevScene &ds = b.scenes[(int)(i - total)];
            const bool on = ds.use_flood && ds.flood_mode != 2;
            ds.flood_counts[0] = 0;
            ds.flood_counts[1] = ds.flood_reuse ? ds.static_counts[1] : 0;
            ds.flood_counts[2] = ds.flood_reuse ? ds.static_counts[2] : (on ? 0 : 1);
            ds.flood_counts[3] = 0;
        }
    }
}

// Batched direct culling of sources: (scene, source, polygon) and then
// (scene, source, tile) warp tasks over the scenes with src_direct.
template <bool ANY_MAPS>
__global__ void k_src_insert_b(const __grid_constant__ BatchDev b) {
    const long long n = b.src_ins_off[b.n];
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w < n;
         w += (gridDim.x * (long long)blockDim.x) >> 5) {
        const int sc = scene_of_b(b.src_ins_off, b.n, w);
        const DevScene &ds = b.scenes[sc];
        const long long e = w - b.src_ins_off[sc];
        const int g = (int)(e / ds.n_poly), q = (int)(e % ds.n_poly);
        if (ANY_MAPS && ds.use_maps) src_insert<true>(ds, g, q, threadIdx.x & 31);
        else src_insert<false>(ds, g, q, threadIdx.x & 31);
    }
}

template <bool ANY_MAPS>
__global__ void k_src_tiles_b(const __grid_constant__ BatchDev b) {
    const long long n = b.src_tile_off[b.n];
    const unsigned gmask = src_group_mask();
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / kSrcGrp; w < n;
         w += (gridDim.x * (long long)blockDim.x) / kSrcGrp) {
        const int sc = scene_of_b(b.src_tile_off, b.n, w);
        const DevScene &ds = b.scenes[sc];
        const int ntiles = ds.tiles_x * ds.tiles_y;
        const long long e = w - b.src_tile_off[sc];
        const int g = (int)(e / ntiles), t = (int)(e % ntiles);
        if (ANY_MAPS && ds.use_maps) src_tile<true>(ds, g, t, threadIdx.x % kSrcGrp, gmask);
        else src_tile<false>(ds, g, t, threadIdx.x % kSrcGrp, gmask);
    }
}

// Exclusive scan of tile_count into tile_start (one CTA), then fill.
// The per-tile CSR of the pairs: the scene's lists, or (to_static) the kept
// lists of the obstacle vertices' flood.
// Each thread scans a run of consecutive tiles, a multiple of four long so
// that a full run moves by 16-byte loads and stores (runs of 16 on the
// 4096^2 maze: four loads instead of sixteen strided ones).
__device__ void tiles_scan_block(const DevScene &ds, bool to_static = false) {
    __shared__ long long wsum[32];
    int32_t *start = to_static ? ds.static_tile_start : ds.tile_start;
    const int n = ds.tiles_x * ds.tiles_y;
    constexpr int kRun = 16;  // vector path: runs of exactly kRun (4 x int4)
    const int per = ((n + blockDim.x - 1) / blockDim.x + 3) & ~3;
    const int lo = threadIdx.x * per, hi = min(n, lo + per);
    const bool vec = per == kRun && hi - lo == kRun;
    int4 c[kRun / 4];
    long long s = 0;
    if (vec) {
#pragma unroll
        for (int k = 0; k < kRun / 4; ++k) {
            c[k] = reinterpret_cast<const int4 *>(ds.tile_count + lo)[k];
            s += (long long)c[k].x + c[k].y + c[k].z + c[k].w;
        }
    } else {
        for (int i = lo; i < hi; ++i) s += ds.tile_count[i];
    }
    long long run = cta_exclusive_scan(s, wsum);  // every thread, once
    if (vec) {
#pragma unroll
        for (int k = 0; k < kRun / 4; ++k) {
            int4 o;
            o.x = (int32_t)run;
            run += c[k].x;
            o.y = (int32_t)run;
            run += c[k].y;
            o.z = (int32_t)run;
            run += c[k].z;
            o.w = (int32_t)run;
            run += c[k].w;
            reinterpret_cast<int4 *>(start + lo)[k] = o;
            reinterpret_cast<int4 *>(ds.tile_count + lo)[k] = make_int4(0, 0, 0, 0);  // reused as fill cursors
        }
    } else {
        for (int i = lo; i < hi; ++i) {
            start[i] = (int32_t)run;
            run += ds.tile_count[i];
            ds.tile_count[i] = 0;  // reused as fill cursor
        }
    }
    if (hi == n && lo < hi) start[n] = (int32_t)run;
    if (threadIdx.x == 0 && n == 0) start[0] = 0;
}

__device__ __forceinline__ void tiles_fill(const DevScene &ds, int i0, int stride, bool to_static = false) {
    const int32_t *start = to_static ? ds.static_tile_start : ds.tile_start;
    int32_t *items = to_static ? ds.static_tile_items : ds.tile_items;
    const int np = min(ds.flood_counts[0], ds.pair_cap);
    for (int i = i0; i < np; i += stride) {
        const int2 pr = ds.pairs[i];
        const int slot = atomicAdd(&ds.tile_count[pr.x], 1);
        items[start[pr.x] + slot] = pr.y;
    }
}

__global__ void __launch_bounds__(1024) k_tiles_scan(DevScene ds, int to_static) { tiles_scan_block(ds, to_static); }

__global__ void k_tiles_fill(DevScene ds, int to_static) {
    tiles_fill(ds, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, to_static);
}

// batched: one CTA per scene for the scan, a row of CTAs per scene for the fill
__global__ void __launch_bounds__(1024) k_tiles_scan_b(const __grid_constant__ BatchDev b) {
    const DevScene &ds = b.scenes[blockIdx.x];
    if (ds.use_flood && ds.flood_mode != 2) tiles_scan_block(ds);
}

__global__ void k_tiles_fill_b(const __grid_constant__ BatchDev b) {
    const DevScene &ds = b.scenes[blockIdx.y];
    if (ds.use_flood && ds.flood_mode != 2) tiles_fill(ds, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

}  // namespace

// dynamic part: visited tiles, inserted polygons, and with maps the lower-bound bins
size_t flood_smem_bytes(int tiles, int polys, bool maps) {
    return sizeof(unsigned) * (size_t)((tiles + 31) / 32 + (polys <= kFloodPolyBits ? (polys + 31) / 32 : 0) +
                                       (maps ? kAng : 0));
}

bool flood_possible(int tiles, int polys) {
    return flood_smem_bytes(tiles, polys, true) + sizeof(FloodSmem) <= 200 * 1024;
}

void launch_flood(const DevScene &ds, cudaStream_t st, FloodStatic how) {
    const int ntiles = ds.tiles_x * ds.tiles_y;
    if (ds.flood_mode == 2) {  // never: the pixel pass scans every generator
        static const int32_t off[4] = {0, 0, 1, 0};
        cudaMemcpyAsync(ds.flood_counts, off, sizeof off, cudaMemcpyHostToDevice, st);
        return;
    }
    const bool maps = ds.use_maps && ds.gen_maps;
    const size_t smem = flood_smem_bytes(ntiles, ds.n_poly, maps);
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, maps ? k_flood<true> : k_flood<false>, kFloodThreads, smem);
    auto flood = [&](int g0, int g1) {
        if (g1 <= g0) return;
        const int blocks = max(1, min(max(sms, 1) * max(per_sm, 1), g1 - g0));  // resident CTAs only
        if (maps) k_flood<true><<<blocks, kFloodThreads, smem, st>>>(ds, g0, g1);
        else k_flood<false><<<blocks, kFloodThreads, smem, st>>>(ds, g0, g1);
    };
    const int sblocks = max(1, min((ntiles + 255) / 256, 152));
    if (how == FloodStatic::kNone) {
        cudaMemsetAsync(ds.tile_count, 0, sizeof(int32_t) * ntiles, st);
        cudaMemsetAsync(ds.flood_counts, 0, sizeof(int32_t) * 4, st);
        flood(0, ds.n_gen);
    } else {
        if (how == FloodStatic::kBuild) {  // the obstacle vertices' lists, kept for every later compute
            cudaMemsetAsync(ds.tile_count, 0, sizeof(int32_t) * ntiles, st);
            cudaMemsetAsync(ds.flood_counts, 0, sizeof(int32_t) * 4, st);
            flood(ds.n_src, ds.n_gen);
            k_tiles_scan<<<1, 1024, 0, st>>>(ds, 1);
            k_tiles_fill<<<152 * 4, 256, 0, st>>>(ds, 1);
            k_flood_static<<<sblocks, 256, 0, st>>>(ds, 1);
        }
        if (flood_sources_direct(ds)) {  // the sources: the only lists a compute sorts
            const int nmap = ds.n_src * kAng;
            k_src_prep<<<max(1, min((max(nmap, ntiles) + 255) / 256, 152 * 4)), 256, 0, st>>>(ds);
            auto wblocks = [](long long warps) { return (int)std::max(1LL, std::min((warps + 7) / 8, 152LL * 16)); };
            if (ds.n_poly > 0) {
                if (maps) k_src_insert<true><<<wblocks((long long)ds.n_src * ds.n_poly), 256, 0, st>>>(ds);
                else k_src_insert<false><<<wblocks((long long)ds.n_src * ds.n_poly), 256, 0, st>>>(ds);
            }
            const long long tgroups = ((long long)ds.n_src * ntiles + 3) / 4;  // warps of four tests
            if (maps) k_src_tiles<true><<<wblocks(tgroups), 256, 0, st>>>(ds);
            else k_src_tiles<false><<<wblocks(tgroups), 256, 0, st>>>(ds);
        } else {
            k_flood_static<<<sblocks, 256, 0, st>>>(ds, 0);
            flood(0, ds.n_src);
        }
    }
    k_tiles_scan<<<1, 1024, 0, st>>>(ds, 0);
    k_tiles_fill<<<152 * 4, 256, 0, st>>>(ds, 0);
}

bool flood_sources_direct(const DevScene &ds) {
    const long long ntiles = (long long)ds.tiles_x * ds.tiles_y;
    return ds.gen_maps && ds.n_src > 0 && (long long)ds.n_src * (ds.n_poly + ntiles) <= (1LL << 24);
}

int flood_smem_attr() {
    const int dyn = 200 * 1024 - (int)sizeof(FloodSmem);
    return cudaFuncSetAttribute(k_flood<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) == cudaSuccess &&
           cudaFuncSetAttribute(k_flood<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) == cudaSuccess &&
           cudaFuncSetAttribute(k_flood_b<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) == cudaSuccess &&
           cudaFuncSetAttribute(k_flood_b<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) == cudaSuccess;
}

void launch_flood_batched(const BatchDev &b, cudaStream_t st, long long src_ins, long long src_tiles) {
    k_flood_reset_b<<<152 * 4, 256, 0, st>>>(b);
    if (b.flood_smem <= 0) return;  // every scene scans
    if (b.walk_tasks > 0) {
        if (b.any_maps) k_flood_b<true><<<152 * 8, kFloodThreads, b.flood_smem, st>>>(b);
        else k_flood_b<false><<<152 * 8, kFloodThreads, b.flood_smem, st>>>(b);
    }
    auto wblocks = [](long long warps) { return (int)std::max(1LL, std::min((warps + 7) / 8, 152LL * 16)); };
    if (src_ins > 0) {
        if (b.any_maps) k_src_insert_b<true><<<wblocks(src_ins), 256, 0, st>>>(b);
        else k_src_insert_b<false><<<wblocks(src_ins), 256, 0, st>>>(b);
    }
    if (src_tiles > 0) {  // four tests per warp
        if (b.any_maps) k_src_tiles_b<true><<<wblocks((src_tiles + 3) / 4), 256, 0, st>>>(b);
        else k_src_tiles_b<false><<<wblocks((src_tiles + 3) / 4), 256, 0, st>>>(b);
    }
    k_tiles_scan_b<<<b.n, 1024, 0, st>>>(b);
    k_tiles_fill_b<<<dim3(16, b.n), 256, 0, st>>>(b);
}

}  // namespace spm

#ifdef SPM_TIME
// Instrumentation build only: reads and clears the flood's phase clocks.
extern "C" int spm_debug_times_flood(unsigned long long *out8) {
    cudaDeviceSynchronize();
    if (cudaMemcpyFromSymbol(out8, spm::g_time, sizeof(unsigned long long) * 8) != cudaSuccess) return 1;
    unsigned long long z[8] = {0};
    cudaMemcpyToSymbol(spm::g_time, z, sizeof z);
    return 0;
}
#endif

#ifdef SPM_COUNT
// Instrumentation build only: reads and clears this unit's work counters.
extern "C" int spm_debug_counters_flood(unsigned long long *out32) {
    cudaDeviceSynchronize();
    if (cudaMemcpyFromSymbol(out32, spm::g_count, sizeof(unsigned long long) * 32) != cudaSuccess) return 1;
    unsigned long long z[32] = {0};
    cudaMemcpyToSymbol(spm::g_count, z, sizeof z);
    return 0;
}
#endif
