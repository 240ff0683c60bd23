// spm_pixel.cu -- pixel phase of the shortest-path map.
//
// arxiv 1805.08500 Sec. 3.1, Procedure 3 ("Cone"): a pixel that sees generator
// g takes cost(g) + |p - g| when that is smaller than what it holds; Sec. 4:
// a segment interior reaches p through its perpendicular foot. Instead of one
// full-screen pass per generator, one CTA owns a 32 x 32 (or 16 x 16) pixel
// tile and gathers only the generators that can win somewhere in it:
//   * free space: the pixels inside obstacles come from the scene's
//     free-space mask (built once, one bit per pixel);
//   * candidates: the tile's list from the flood, or every generator;
//   * cull: finite cost, shadow cone (or perpendicular strip) meets the tile,
//     lower bound lb = cost + dist(g, tile) below the tile's current worst;
//   * order: candidates sorted by lb; the CTA stops once every pixel's best is
//     <= lb (no later candidate can win);
//   * hidden tiles: in lb order, in chunks of 32, 64, 128, then 256
//     candidates (the early exit usually comes within the first chunk), each
//     thread walks
//     the polygon bins from the tile toward one candidate and drops it when a
//     single polygon hides all four corners of the tile (the region a convex
//     polygon hides from a point is convex, so the whole tile is hidden);
//   * depth maps (when the flood kept them): a pixel nearer than the lower
//     bound of its bin sees the candidate, one beyond the full-blocking upper
//     bound does not; only the pixels in between take the exact test below;
//   * visibility: for each candidate still useful to some pixel, the CTA
//     builds the list of polygons whose interior meets the hull of (tile, g)
//     (exact separating-axis filter), then every pixel runs the exact integer
//     separating-axis test against that list (none when the list is empty);
//   * argmin: a per-pixel u64 key (FP32 distance bits << 32 | generator id),
//     so "smaller distance, then smaller id" is one unsigned compare;
//   * output: each thread owns 4 consecutive pixels of a row and writes them
//     with one 16-byte store per plane (dist, parent).
#include <cuda_runtime.h>

#include "spm_device.cuh"
#include "spm_internal.h"

namespace spm {
namespace {

constexpr int NT = kPixelThreads;
#ifndef SPM_PIX16_MINB
#define SPM_PIX16_MINB 4  // resident CTAs per SM the 16 x 16 kernel is compiled for
#endif
#ifndef SPM_PIX32_MINB
#define SPM_PIX32_MINB 4  // the same for the 32 x 32 kernel
#endif
#ifndef SPM_PIXB_MINB
#define SPM_PIXB_MINB 3   // the same for the batched kernel (both tile sizes inlined)
#endif
constexpr unsigned long long kUnset = 0x7F800000FFFFFFFFull;  // (+inf, id max)

// Work counters of an instrumentation build (-DSPM_COUNT); compiled out otherwise.


// Convex hull (counter-clockwise, no repeated or collinear vertices) of the
// tile's pixel-centre box and the lattice point t, by Andrew's monotone chain
// over the 5 points. The box may be degenerate (a one-pixel row or column),
// so the hull may be a segment (2 vertices) or a point (1).
struct Hull {
    int2 v[5];
    int n;
};

__device__ __forceinline__ Hull hull_box_point(int4 box, int tx, int ty) {
    int2 p[5] = {make_int2(box.x, box.y), make_int2(box.z, box.y), make_int2(box.z, box.w), make_int2(box.x, box.w),
                 make_int2(tx, ty)};
#pragma unroll
    for (int i = 1; i < 5; ++i)  // sort by (x, y)
#pragma unroll
        for (int j = i; j > 0; --j)
            if (p[j].x < p[j - 1].x || (p[j].x == p[j - 1].x && p[j].y < p[j - 1].y)) {
                const int2 t = p[j];
                p[j] = p[j - 1];
                p[j - 1] = t;
            }
    int2 st[10];
    int k = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i) {  // lower chain
        while (k >= 2 && orient32(st[k - 2].x, st[k - 2].y, st[k - 1].x, st[k - 1].y, p[i].x, p[i].y) <= 0) --k;
        st[k++] = p[i];
    }
    const int lower = k + 1;
#pragma unroll
    for (int i = 3; i >= 0; --i) {  // upper chain
        while (k >= lower && orient32(st[k - 2].x, st[k - 2].y, st[k - 1].x, st[k - 1].y, p[i].x, p[i].y) <= 0) --k;
        st[k++] = p[i];
    }
    Hull h;
    h.n = k > 1 ? k - 1 : 1;  // the last point repeats the first
    if (h.n == 2 && st[0].x == st[1].x && st[0].y == st[1].y) h.n = 1;
#pragma unroll
    for (int i = 0; i < 5; ++i) h.v[i] = st[i < h.n ? i : 0];
    return h;
}

// Per-candidate generator data staged in shared memory for the first
// kStage candidates of a sorted batch: one parallel load replaces a dependent
// global load per candidate in the lb-ordered loop.
constexpr int kStage = 64;
struct CandRec {
    int4 cone;
    int2 lat;
    float2 pos;
    float cf;
    int kind, ctype, map_ok;
};

struct PixSmem {
    CandRec rec[kStage];
    int cand_id[kCandCap];
    float cand_lb[kCandCap];
    unsigned dedup[kDedupBits / 32];
    int2 blk_v[kBlockCap][kMaxPolyVerts];
    int blk_oA[kBlockCap][kMaxPolyVerts];
    int blk_oB[kBlockCap][kMaxPolyVerts];
    unsigned blk_mask[kBlockCap];
    int blk_m[kBlockCap];
    unsigned char hidden[kCandCap];
    int n_cand, n_block, overflow;
    float tile_ub;
    Hull hull;  // of the tile box and the current point target
};

// Does the interior of convex polygon V meet the closed convex hull H?
// Separating-axis test over the edges of both (an edge separates when the
// other body lies on its closed outer side).
__device__ bool poly_meets_hull(const int2 *V, int m, const Hull &H) {
    for (int i = 0; i < m; ++i) {  // polygon edges (outward side is orient < 0)
        const int2 a = V[i], b = V[i + 1 == m ? 0 : i + 1];
        bool all_out = true;
        for (int k = 0; k < H.n && all_out; ++k) all_out = orient32(a.x, a.y, b.x, b.y, H.v[k].x, H.v[k].y) <= 0;
        if (all_out) return false;
    }
    for (int j = 0; j < H.n; ++j) {  // hull edges
        const int2 a = H.v[j], b = H.v[j + 1 == H.n ? 0 : j + 1];
        if (a.x == b.x && a.y == b.y) continue;  // a one-point hull has no edge
        bool all_out = true;
        for (int i = 0; i < m && all_out; ++i) all_out = orient32(a.x, a.y, b.x, b.y, V[i].x, V[i].y) <= 0;
        if (all_out) return false;
    }
    return true;
}

__device__ __forceinline__ float key_dist(unsigned long long k) { return __uint_as_float((unsigned)(k >> 32)); }

// Lower bound of cost(g) + distance from g to any pixel of the tile, or -1 if
// g cannot be valid anywhere in the tile.
__device__ float tile_lower_bound(const DevScene &ds, int g, int4 box, float4 fbox) {
    // every field is loaded up front (independent loads, in flight together)
    const float cf = __ldg(ds.gen_costf + g);
    const int kind = __ldg(ds.gen_kind + g);
    const int ctype = __ldg(ds.gen_ctype + g);
    const int4 cone = __ldg(ds.gen_cone + g);
    const int2 gv = __ldg(ds.gen_lat + g);
    const float2 gpos = __ldg(ds.gen_pos + g);
    if (!(cf < INFINITY)) return -1.f;
    if (kind == kSegI) {
        const int s = ds.gen_aux[g];
        const int4 L = ds.seg_lat[s];
        const long long ux = L.z - L.x, uy = L.w - L.y, den = ux * ux + uy * uy;
        bool all_lo = true, all_hi = true;
        const int cx[4] = {box.x, box.z, box.x, box.z}, cy[4] = {box.y, box.y, box.w, box.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            long long num = (cx[k] - L.x) * ux + (cy[k] - L.y) * uy;
            all_lo &= num <= 0;
            all_hi &= num >= den;
        }
        if (all_lo || all_hi) return -1.f;
        const float4 F = ds.seg_pos[s];
        const float fx = F.z - F.x, fy = F.w - F.y, il = rsqrtf(fx * fx + fy * fy);
        const float qx[4] = {fbox.x, fbox.z, fbox.x, fbox.z}, qy[4] = {fbox.y, fbox.y, fbox.w, fbox.w};
        float mn = INFINITY;
        bool pos = false, neg = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float sd = (fx * (qy[k] - F.y) - fy * (qx[k] - F.x)) * il;
            pos |= sd > 0.f;
            neg |= sd < 0.f;
            mn = fminf(mn, fabsf(sd));
        }
        return (pos && neg) ? 0.f : mn * 0.999999f;
    }
    if (kind == kVert) {
        const int ct = ctype;
        if (ct == kConeEmpty) return -1.f;
        const int4 c = cone;
        const int2 v = gv;
        const int cx[4] = {box.x, box.z, box.x, box.z}, cy[4] = {box.y, box.y, box.w, box.w};
        bool out1 = true, out2 = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int wx = cx[k] - v.x, wy = cy[k] - v.y;
            out1 &= cross32(c.x, c.y, wx, wy) < 0;
            out2 &= cross32(wx, wy, c.z, c.w) < 0;
        }
        if (out1 || out2) return -1.f;
    }
    const float2 p = gpos;
    const float dx = fmaxf(fmaxf(fbox.x - p.x, p.x - fbox.z), 0.f);
    const float dy = fmaxf(fmaxf(fbox.y - p.y, p.y - fbox.w), 0.f);
    return (cf + sqrtf(dx * dx + dy * dy)) * 0.999999f;
}

// Bitonic sort of (lb, id) pairs, n padded to a power of two with +inf
// (lists of more than 32; shorter ones take sort_small_warp).
__device__ void sort_candidates(PixSmem &sm, int n) {
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = n + threadIdx.x; i < P; i += NT) {
        sm.cand_lb[i] = INFINITY;
        sm.cand_id[i] = 0x7fffffff;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += NT) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const float a = sm.cand_lb[i], b = sm.cand_lb[ixj];
                    const int ia = sm.cand_id[i], ib = sm.cand_id[ixj];
                    const bool gt = (a > b) || (a == b && ia > ib);
                    if (gt == up) {
                        sm.cand_lb[i] = b; sm.cand_lb[ixj] = a;
                        sm.cand_id[i] = ib; sm.cand_id[ixj] = ia;
                    }
                }
            }
            __syncthreads();
        }
}

// The generator data the candidate loop reads, staged in shared memory.
template <bool MAPS>
__device__ __forceinline__ CandRec stage_candidate(const DevScene &ds, int g) {
    CandRec r;
    r.kind = ds.gen_kind[g];
    r.cf = ds.gen_costf[g];
    r.lat = ds.gen_lat[g];
    r.pos = ds.gen_pos[g];
    r.ctype = r.kind == kVert ? ds.gen_ctype[g] : kConeNone;
    r.cone = r.kind == kVert ? ds.gen_cone[g] : make_int4(0, 0, 0, 0);
    r.map_ok = MAPS && ds.gen_map_ok ? ds.gen_map_ok[g] : 0;
    return r;
}

// Up to 32 (lb, id) pairs, nearly every tile's list, sorted by the first warp
// in registers with shuffles (a bitonic network of the next power of two
// above n), each lane then staging its candidate's generator data; the CTA
// waits once.
template <bool MAPS>
__device__ void sort_small_warp(const DevScene &ds, PixSmem &sm, int n) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        float lb = lane < n ? sm.cand_lb[lane] : INFINITY;
        int id = lane < n ? sm.cand_id[lane] : 0x7fffffff;
        int P = 1;
        while (P < n) P <<= 1;
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                const float olb = __shfl_xor_sync(0xffffffffu, lb, j);
                const int oid = __shfl_xor_sync(0xffffffffu, id, j);
                // the lower lane of a pair keeps the smaller key in an
                // ascending run ((lane & k) == 0), the larger otherwise
                const bool lower = (lane & j) == 0, up = (lane & k) == 0;
                const bool o_less = olb < lb || (olb == lb && oid < id);
                if (o_less == (lower == up)) {
                    lb = olb;
                    id = oid;
                }
            }
        if (lane < n) {
            sm.cand_lb[lane] = lb;
            sm.cand_id[lane] = id;
            sm.rec[lane] = stage_candidate<MAPS>(ds, id);  // kStage >= 32
        }
    }
    __syncthreads();
}

// Conservative bin enumeration for the thick segment c->t (lattice units,
// radius r): column-wise, one (column, bin) item per thread, so that every
// thread scans one bin's records. Each polygon found is filtered against the
// thick segment and appended (deduplicated) to smem.
__device__ void build_blockers(const DevScene &ds, PixSmem &sm, float cx, float cy, float tx, float ty,
                               float r, int kind, int2 tl, int4 seg, int4 box) {
    // Float steps here only choose bins; their errors (~1e-3 lattice units)
    // stay far inside the margin m, so fast reciprocals are safe.
    const float bs = (float)ds.bin_size, ibs = 1.0f / bs, x0 = (float)ds.bin_x0, y0 = (float)ds.bin_y0;
    const float m = r + 1.0f;
    auto bin_of = [&](float v, float o, int n) {
        int b = (int)floorf((v - o) * ibs);
        return b < 0 ? 0 : (b >= n ? n - 1 : b);
    };
    const int c0 = bin_of(fminf(cx, tx) - m, x0, ds.bin_nx), c1 = bin_of(fmaxf(cx, tx) + m, x0, ds.bin_nx);
    const float dx = tx - cx, dy = ty - cy;
    const bool dedup = ds.n_poly <= kDedupBits;
    // items per column: about the rows one column spans (its x extent is
    // bs + 2m, the segment rises |dy/dx| per unit along it, plus m on both
    // sides); each item strides by K, so any K covers every row
    const float idx = fabsf(dx) < 0.5f ? 0.f : __fdividef(1.0f, dx);
    const float span = fabsf(dx) < 0.5f ? fabsf(dy) + 2.f * m : fabsf(dy * idx) * (bs + 2.f * m) + 2.f * m;
    const int K = min((int)(span * ibs) + 2, ds.bin_ny);
    const int items = (c1 - c0 + 1) * K;
    for (int j = threadIdx.x; j < items; j += NT) {
        const int col = c0 + j / K, kr = j - (j / K) * K;
        float ylo, yhi;
        if (fabsf(dx) < 0.5f) {
            ylo = fminf(cy, ty);
            yhi = fmaxf(cy, ty);
        } else {
            float a = x0 + col * bs - m, b = x0 + (col + 1) * bs + m;
            float t0 = (a - cx) * idx, t1 = (b - cx) * idx;
            float tlo = fmaxf(0.f, fminf(t0, t1)), thi = fminf(1.f, fmaxf(t0, t1));
            if (tlo > thi) { tlo = 0.f; thi = 1.f; }
            float ya = cy + tlo * dy, yb = cy + thi * dy;
            ylo = fminf(ya, yb);
            yhi = fmaxf(ya, yb);
        }
        const int r0 = bin_of(ylo - m, y0, ds.bin_ny), r1 = bin_of(yhi + m, y0, ds.bin_ny);
        for (int row = r0 + kr; row <= r1; row += K) {  // rows kr, kr + K, ...: every row once
            const int bin = row * ds.bin_nx + col;
            const int e = __ldg(ds.bin_start + bin + 1);
            for (int it = __ldg(ds.bin_start + bin); it < e; ++it) {
                const int4 *rp = reinterpret_cast<const int4 *>(ds.bin_recs + it);
                const BinRec rec = {__ldg(rp), __ldg(rp + 1).x, __ldg(rp + 1).y, __ldg(rp + 1).z, 0};
                const int k = rec.poly;
                if (dedup) {
                    const unsigned bit = 1u << (k & 31);
                    if (atomicOr(&sm.dedup[k >> 5], bit) & bit) continue;
                }
                if (!seg_near_box(cx, cy, tx, ty, r, rec.box)) continue;
                if (kind != kSegI && !poly_meets_hull(ds.poly_v + rec.voff, rec.m, sm.hull)) continue;
                const int slot = atomicAdd(&sm.n_block, 1);
                if (slot >= kBlockCap) {
                    sm.overflow = 1;
                    continue;
                }
                const int b = rec.voff, nv = rec.m;
                sm.blk_m[slot] = nv;
                for (int i = 0; i < nv; ++i) sm.blk_v[slot][i] = ds.poly_v[b + i];
                if (kind == kSegI) {
                    for (int i = 0; i < nv; ++i) {
                        const int2 a = sm.blk_v[slot][i], bb = sm.blk_v[slot][i + 1 == nv ? 0 : i + 1];
                        sm.blk_oA[slot][i] = orient32(a.x, a.y, bb.x, bb.y, seg.x, seg.y);
                        sm.blk_oB[slot][i] = orient32(a.x, a.y, bb.x, bb.y, seg.z, seg.w);
                    }
                } else {
                    sm.blk_mask[slot] = edge_mask(sm.blk_v[slot], nv, tl.x, tl.y);
                }
            }
        }
    }
}

// One tile of one scene, by one CTA: 32 x 32 pixels with PX = 4 pixels per
// thread (consecutive in a row), or 16 x 16 with PX = 1. allow_lists = false
// ignores flooded candidate lists (the batched form scans every generator).
template <int PX, bool MAPS>
__device__ __forceinline__ void pixel_tile(const DevScene &ds, const int tile, float *__restrict__ dist,
                                           int32_t *__restrict__ parent, PixSmem &sm, const bool allow_lists) {
    constexpr int T = PX == 4 ? 32 : 16;
    constexpr int TPR = T / PX;  // threads per tile row
    SPM_T0();
    const int i0 = (tile % ds.tiles_x) * T, j0 = (tile / ds.tiles_x) * T;
    const int row = threadIdx.x / TPR, c4 = (threadIdx.x % TPR) * PX;
    const int j = j0 + row;
    const int pitch_x = ds.S * ds.Wx / ds.Nx, pitch_y = ds.S * ds.Wy / ds.Ny;
    const int py = pitch_y * j + pitch_y / 2;
    const float fy = ((float)j + 0.5f) * ds.hy;
    int px[PX];
    float fx[PX];
    unsigned long long key[PX];
    unsigned live = 0;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const int i = i0 + c4 + k;
        px[k] = pitch_x * i + pitch_x / 2;
        fx[k] = ((float)i + 0.5f) * ds.hx;
        key[k] = kUnset;
        if (i < ds.Nx && j < ds.Ny) live |= 1u << k;
    }
    // free space: not in the open interior of any polygon (the scene's
    // free-space mask; the PX pixels of a thread share one word)
    if (j < ds.Ny) {
        const uint32_t fw = __ldg(ds.free_bits + (size_t)j * ds.free_words + ((i0 + c4) >> 5));
#pragma unroll
        for (int k = 0; k < PX; ++k)
            if (!((fw >> ((i0 + c4 + k) & 31)) & 1u)) live &= ~(1u << k);
    }
    const int ni = min(T, ds.Nx - i0), nj = min(T, ds.Ny - j0);
    const int4 box = make_int4(pitch_x * i0 + pitch_x / 2, pitch_y * j0 + pitch_y / 2,
                               pitch_x * (i0 + ni - 1) + pitch_x / 2, pitch_y * (j0 + nj - 1) + pitch_y / 2);
    const float4 fbox = make_float4(((float)i0 + 0.5f) * ds.hx, ((float)j0 + 0.5f) * ds.hy,
                                    ((float)(i0 + ni - 1) + 0.5f) * ds.hx, ((float)(j0 + nj - 1) + 0.5f) * ds.hy);
    const float bcx = 0.5f * ((float)box.x + (float)box.z), bcy = 0.5f * ((float)box.y + (float)box.w);
    const float brad = 0.5f * sqrtf((float)(box.z - box.x) * (float)(box.z - box.x) +
                                    (float)(box.w - box.y) * (float)(box.w - box.y)) + 1.0f;
    const bool any_live = __syncthreads_or(live != 0);
    if (threadIdx.x == 0) SPM_CNT(0, 1);
    if (threadIdx.x == 0) {
        sm.n_cand = 0;
        sm.tile_ub = INFINITY;
    }
    __syncthreads();
    SPM_LAP(0);
    // candidate source: the tile's flooded lists (the obstacle vertices' kept
    // list, when this compute reuses it, then this flood's list) plus the
    // global list, or every generator when the lists are unavailable
    const bool lists = allow_lists && ds.use_flood && ds.flood_counts[2] == 0;
    const bool stat = lists && ds.static_lists;
    const int tix = tile;
    const int s0 = stat ? ds.static_tile_start[tix] : 0;
    const int ns = stat ? ds.static_tile_start[tix + 1] - s0 : 0;
    const int l0 = lists ? ds.tile_start[tix] : 0;
    const int nl = ns + (lists ? ds.tile_start[tix + 1] - l0 : 0);
    const int ntotal = lists ? nl + ds.flood_counts[1] : ds.n_gen;
    for (int g0 = 0; any_live && g0 < ntotal; g0 += NT) {
        const int i = g0 + threadIdx.x;
        int g = i;
        if (lists && i < ntotal)
            g = i < ns ? ds.static_tile_items[s0 + i] : i < nl ? ds.tile_items[l0 + i - ns] : ds.glob_list[i - nl];
        float lb = -1.f;
        if (i < ntotal) lb = tile_lower_bound(ds, g, box, fbox);
        const bool keep = lb >= 0.f && lb <= sm.tile_ub;
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        int base = 0;
        if ((threadIdx.x & 31) == 0 && bal) base = atomicAdd(&sm.n_cand, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) {
            const int slot = base + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u));
            sm.cand_id[slot] = g;
            sm.cand_lb[slot] = lb;
        }
        __syncthreads();
        SPM_LAP(1);
        const int nc = sm.n_cand;
        const bool last = g0 + NT >= ntotal;
        if (nc > kCandCap - NT || (last && nc > 0)) {
            static_assert(kStage >= 32, "a warp-sorted list is staged whole");
            if (nc <= 32) {
                sort_small_warp<MAPS>(ds, sm, nc);
            } else {
                sort_candidates(sm, nc);
                for (int t = threadIdx.x; t < min(nc, kStage); t += NT) sm.rec[t] = stage_candidate<MAPS>(ds, sm.cand_id[t]);
                __syncthreads();
            }
            SPM_LAP(2);
            if (threadIdx.x == 0) SPM_CNT(1, nc);
            bool done = false;
            int tested = 0, chunk = ds.hidden_chunk;
            for (int c = 0; c < nc && !done; ++c) {
                const float lb_c = sm.cand_lb[c];
                bool act = false;
#pragma unroll
                for (int k = 0; k < PX; ++k) act |= (live >> k & 1u) && key_dist(key[k]) > lb_c;
                if (!__syncthreads_or(act)) {
                    done = true;
                    SPM_LAP(3);
                    break;
                }
                SPM_LAP(3);
                // flooded lists were already tested on the whole tile area:
                // no hidden-tile tests (nor their barriers) with lists
                if (!lists && c == tested) {  // hidden-tile test for the next chunk, in parallel
                    const int cc = c + threadIdx.x;
                    if (threadIdx.x < chunk && cc < nc) {
                        SPM_CNT(2, 1);
                        const int g2 = sm.cand_id[cc];
                        sm.hidden[cc] = ds.gen_kind[g2] != kSegI && box_hidden(ds, ds.gen_lat[g2], box, bcx, bcy, brad);
                    }
                    tested += chunk;
                    chunk = min(2 * chunk, NT);  // most tiles exit within the first chunk
                    __syncthreads();
                }
                if (!lists && sm.hidden[c]) {
                    if (threadIdx.x == 0) SPM_CNT(3, 1);
                    continue;
                }
                if (threadIdx.x == 0) SPM_CNT(4, 1);
                const int gc = sm.cand_id[c];
                const bool staged = c < kStage;
                const int kind = staged ? sm.rec[c].kind : ds.gen_kind[gc];
                const float cf = staged ? sm.rec[c].cf : ds.gen_costf[gc];
                const int2 gl = staged ? sm.rec[c].lat : ds.gen_lat[gc];
                const float2 gp = staged ? sm.rec[c].pos : ds.gen_pos[gc];
                int ct = kConeNone;
                int4 cone = make_int4(0, 0, 0, 0);
                int4 seg = make_int4(0, 0, 0, 0);
                float4 segf = make_float4(0.f, 0.f, 0.f, 0.f);
                long long den = 0;
                float seg_il = 0.f;
                if (kind == kVert) {
                    ct = staged ? sm.rec[c].ctype : ds.gen_ctype[gc];
                    cone = staged ? sm.rec[c].cone : ds.gen_cone[gc];
                } else if (kind == kSegI) {
                    seg = ds.seg_lat[ds.gen_aux[gc]];
                    segf = ds.seg_pos[ds.gen_aux[gc]];
                    const long long ux = seg.z - seg.x, uy = seg.w - seg.y;
                    den = ux * ux + uy * uy;
                    const float fux = segf.z - segf.x, fuy = segf.w - segf.y;
                    seg_il = 1.0f / sqrtf(fux * fux + fuy * fuy);
                }
                unsigned need = 0, want = 0;
                unsigned long long nk[PX];
                long long num[PX];
                // the flood's depth map of a point generator decides most pixels:
                // nearer than any obstacle on their ray -> visible; beyond a full
                // blocking -> hidden; only the rest need the exact test below
                const float2 *gmap = MAPS && lists && ds.use_maps && ds.gen_maps && kind != kSegI &&
                                             (staged ? sm.rec[c].map_ok : ds.gen_map_ok[gc])
                                         ? ds.gen_maps + (size_t)gc * kAngBins
                                         : nullptr;
                // first pass: each pixel's key and depth-map bins, without
                // branches around the loads, so that all of the thread's map
                // loads are in flight together
                float r2[PX];
                int bA[PX], bB[PX];
#pragma unroll
                for (int k = 0; k < PX; ++k) {
                    bool ok = ((live >> k) & 1u) && key_dist(key[k]) > lb_c;
                    float d;
                    num[k] = 0;
                    if (kind == kSegI) {
                        const long long nm = (long long)(px[k] - seg.x) * (seg.z - seg.x) +
                                             (long long)(py - seg.y) * (seg.w - seg.y);
                        ok = ok && nm > 0 && nm < den;
                        num[k] = nm;
                        d = fabsf((segf.z - segf.x) * (fy - segf.y) - (segf.w - segf.y) * (fx[k] - segf.x)) * seg_il;
                    } else {
                        ok = ok && (kind != kVert || in_cone(ct, cone, px[k] - gl.x, py - gl.y));
                        const float ddx = fx[k] - gp.x, ddy = fy - gp.y;
                        d = cf + sqrtf(ddx * ddx + ddy * ddy);
                    }
                    nk[k] = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)gc;
                    if (ok && nk[k] < key[k]) want |= 1u << k;
                    const int rx = px[k] - gl.x, ry = py - gl.y;
                    // float products (|rx|, |ry| < 2^15: relative error below 2^-22,
                    // inside the 1e-5 margins of the map tests below)
                    r2[k] = fmaf((float)rx, (float)rx, (float)ry * (float)ry);
                    const float a = (rx | ry) ? pang((float)rx, (float)ry) : 0.f;
                    bA[k] = ((int)floorf((a - kAngEps) / kAngW) + kAngBins) & (kAngBins - 1);
                    bB[k] = (int)floorf((a + kAngEps) / kAngW) & (kAngBins - 1);
                }
                if (MAPS && gmap) {
                    float2 m0[PX], m1[PX];
#pragma unroll
                    for (int k = 0; k < PX; ++k) {
                        m0[k] = make_float2(0.f, 0.f);
                        m1[k] = m0[k];
                        if ((want >> k) & 1u) {
                            m0[k] = __ldg(gmap + bA[k]);
                            m1[k] = __ldg(gmap + bB[k]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < PX; ++k) {
                        if (!((want >> k) & 1u)) continue;
                        SPM_CNT(14, 1);  // a pixel-candidate pair that needs a visibility decision
                        if (px[k] == gl.x && py == gl.y) {  // the generator's own pixel
                            key[k] = nk[k];
                            continue;
                        }
                        if (r2[k] * (1.f - 1e-5f) >= fmaxf(m0[k].x, m1[k].x)) {  // hidden
                            SPM_CNT(13, 1);
                            continue;
                        }
                        if (r2[k] * (1.f + 1e-5f) < fminf(m0[k].y, m1[k].y)) {  // visible
                            SPM_CNT(12, 1);
                            key[k] = nk[k];
                            continue;
                        }
                        need |= 1u << k;
                    }
                } else {
                    need = want;
                    SPM_CNT(14, __popc(want));
                }
                if (!__syncthreads_or(need != 0)) {
                    SPM_LAP(4);
                    continue;
                }
                SPM_LAP(4);
                if (threadIdx.x == 0) SPM_CNT(5, 1);
                // blockers of the hull of (tile, target)
                float tx, ty;
                if (kind == kSegI) {
                    const float ux = (float)(seg.z - seg.x), uy = (float)(seg.w - seg.y);
                    const float t = ((bcx - seg.x) * ux + (bcy - seg.y) * uy) / (ux * ux + uy * uy);
                    tx = seg.x + t * ux;
                    ty = seg.y + t * uy;
                } else {
                    tx = (float)gl.x;
                    ty = (float)gl.y;
                }
                for (int w = threadIdx.x; w < kDedupBits / 32; w += NT) sm.dedup[w] = 0u;
                if (threadIdx.x == 0) {
                    sm.n_block = 0;
                    sm.overflow = 0;
                    if (kind != kSegI) sm.hull = hull_box_point(box, gl.x, gl.y);
                }
                __syncthreads();
                build_blockers(ds, sm, bcx, bcy, tx, ty, brad, kind, gl, seg, box);
                __syncthreads();
                SPM_LAP(5);
                const int nb = min(sm.n_block, kBlockCap);
                const bool ovf = sm.overflow != 0;
                if (threadIdx.x == 0) {
                    SPM_CNT(6, nb);
                    SPM_CNT(8, ovf ? 1 : 0);
                    if (nb == 0) SPM_CNT(9, 1);
                }
                SPM_CNT(7, __popc(need));
                const int nx = -(seg.w - seg.y), ny = seg.z - seg.x;
#pragma unroll
                for (int k = 0; k < PX; ++k) {
                    if (!((need >> k) & 1u)) continue;
                    bool vis;
                    if (ovf) {
                        vis = kind == kSegI ? visible_foot(ds, ds.gen_aux[gc], px[k], py, num[k], den)
                                            : visible_points(ds, px[k], py, gl.x, gl.y);
                    } else if (kind == kSegI) {
                        vis = true;
                        if (cross32(seg.z - seg.x, seg.w - seg.y, px[k] - seg.x, py - seg.y) != 0)
                            for (int b = 0; b < nb && vis; ++b)
                                vis = !poly_blocks_foot(sm.blk_v[b], sm.blk_m[b], sm.blk_oA[b], sm.blk_oB[b],
                                                        px[k], py, num[k], den, nx, ny);
                    } else {
                        vis = true;
                        if (px[k] != gl.x || py != gl.y)
                            for (int b = 0; b < nb && vis; ++b)
                            {
                                vis = !poly_blocks(sm.blk_v[b], sm.blk_m[b], px[k], py, gl.x, gl.y, sm.blk_mask[b]);
                                SPM_CNT(10, 1);
                                SPM_CNT(11, sm.blk_m[b]);  // orientations of the polygon's edge pass
                            }
                    }
                    if (vis) key[k] = nk[k];
                }
                __syncthreads();
                SPM_LAP(6);
            }
            // tile upper bound for the next batch's candidate pruning (worst
            // best over live pixels); after the last batch nothing reads it
            if (!last) {
                float worst = 0.f;
#pragma unroll
                for (int k = 0; k < PX; ++k)
                    if ((live >> k) & 1u) worst = fmaxf(worst, key_dist(key[k]));
                for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
                __syncthreads();
                if (threadIdx.x == 0) {
                    sm.n_cand = 0;
                    sm.tile_ub = 0.f;
                }
                __syncthreads();
                if ((threadIdx.x & 31) == 0) atomicMax((int *)&sm.tile_ub, __float_as_int(worst));
                __syncthreads();
            }
        }
    }

    if (j < ds.Ny) {
        float od[PX];
        int op[PX];
#pragma unroll
        for (int k = 0; k < PX; ++k) {
            const bool ok = ((live >> k) & 1u) && key[k] != kUnset;
            od[k] = ok ? key_dist(key[k]) : INFINITY;
            op[k] = ok ? (int)(unsigned)(key[k] & 0xffffffffu) : -1;
        }
        const size_t base = (size_t)j * ds.Nx + i0 + c4;
        if (PX == 4 && (ds.Nx & 3) == 0 && i0 + c4 + 3 < ds.Nx) {
            *reinterpret_cast<float4 *>(dist + base) = make_float4(od[0], od[PX > 1 ? 1 : 0], od[PX > 2 ? 2 : 0], od[PX > 3 ? 3 : 0]);
            *reinterpret_cast<int4 *>(parent + base) = make_int4(op[0], op[PX > 1 ? 1 : 0], op[PX > 2 ? 2 : 0], op[PX > 3 ? 3 : 0]);
        } else {
            for (int k = 0; k < PX; ++k)
                if (i0 + c4 + k < ds.Nx) {
                    dist[base + k] = od[k];
                    parent[base + k] = op[k];
                }
        }
    }
    SPM_LAP(7);
    SPM_TFLUSH();
}

// One CTA per tile; one kernel per tile size, so each gets its own register
// allocation (32 x 32 tiles: 4 pixels a thread, 16 x 16: 1).
template <int PX, bool MAPS>
__global__ void __launch_bounds__(NT, PX == 4 ? SPM_PIX32_MINB : SPM_PIX16_MINB) k_pixels(const __grid_constant__ DevScene ds,
                                                                         float *__restrict__ dist,
                                                                         int32_t *__restrict__ parent, int tile0) {
    __shared__ PixSmem sm;
    pixel_tile<PX, MAPS>(ds, tile0 + blockIdx.x, dist, parent, sm, true);
}

// Persistent form over a batch of scenes: each CTA takes the next
// (scene, tile) from a global counter (costliest tiles first), copies
// that scene's descriptor into shared memory and runs the same tile code.
template <bool ANY_MAPS>  // some scene of the batch uses depth maps
__global__ void __launch_bounds__(NT, SPM_PIXB_MINB) k_pixels_batched(const __grid_constant__ BatchDev b) {
    __shared__ PixSmem sm;
    __shared__ DevScene sds;
    __shared__ int cur, cur_scene;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(b.tile_counter, 1);
            cur = t;
            if (t < b.total_tiles) {
                int lo = 0, hi = b.n;  // last order index with tile_off <= t
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (b.tile_off[mid] <= t) lo = mid;
                    else hi = mid;
                }
                cur_scene = lo;
            }
        }
        __syncthreads();
        const int t = cur;
        if (t >= b.total_tiles) break;
        const int oi = cur_scene, sc = b.order[oi];
        for (int w = threadIdx.x; w < (int)(sizeof(DevScene) / 4); w += NT)
            reinterpret_cast<int *>(&sds)[w] = reinterpret_cast<const int *>(&b.scenes[sc])[w];
        __syncthreads();
        if (sds.tile == kTile) pixel_tile<4, ANY_MAPS>(sds, t - b.tile_off[oi], b.dist[sc], b.parent[sc], sm, true);
        else pixel_tile<1, ANY_MAPS>(sds, t - b.tile_off[oi], b.dist[sc], b.parent[sc], sm, true);
        __syncthreads();
    }
}

}  // namespace

// Exact point query (Sec. 6, Discussion: a point on a region border may take
// a parent up to half a pixel's diagonal off; comparing the parents of the
// neighbouring pixels at the point itself removes the error). One warp: lane
// k < 9 evaluates the parent of pixel (i + k % 3 - 1, j + k / 3 - 1) at the
// lattice point q (world coordinates qf) with the exact predicates, FP64 keys
// in the same operation order as the distance definition; the smallest key
// (then id) wins.
__global__ void k_query_exact(const __grid_constant__ DevScene ds, const int32_t *__restrict__ field_parent, int i,
                              int j, int2 q, double2 qf, int32_t *out_par, double *out_dist) {
    const int lane = threadIdx.x;
    int g = -1;
    if (lane < 9) {
        const int ii = i + lane % 3 - 1, jj = j + lane / 3 - 1;
        if (ii >= 0 && jj >= 0 && ii < ds.Nx && jj < ds.Ny) g = field_parent[(size_t)jj * ds.Nx + ii];
    }
    double key = INFINITY;
    if (g >= 0 && ds.gen_cost[g] < INFINITY) {
        const int kind = ds.gen_kind[g];
        if (kind == kSegI) {
            const int s = ds.gen_aux[g];
            const int4 L = ds.seg_lat[s];
            const long long ux = L.z - L.x, uy = L.w - L.y;
            const long long num = (q.x - L.x) * ux + (q.y - L.y) * uy, den = ux * ux + uy * uy;
            if (num > 0 && num < den && visible_foot(ds, s, q.x, q.y, num, den)) {
                const float4 F = ds.seg_pos[s];
                const double fx = __dsub_rn((double)F.z, (double)F.x), fy = __dsub_rn((double)F.w, (double)F.y);
                const double c = __dsub_rn(__dmul_rn(fx, __dsub_rn(qf.y, (double)F.y)), __dmul_rn(fy, __dsub_rn(qf.x, (double)F.x)));
                key = __ddiv_rn(fabs(c), __dsqrt_rn(__dadd_rn(__dmul_rn(fx, fx), __dmul_rn(fy, fy))));
            }
        } else {
            const int2 gl = ds.gen_lat[g];
            const bool cone_ok = kind != kVert || in_cone(ds.gen_ctype[g], ds.gen_cone[g], q.x - gl.x, q.y - gl.y);
            if (cone_ok && visible_points(ds, q.x, q.y, gl.x, gl.y)) {
                const float2 gp = ds.gen_pos[g];
                const double dx = __dsub_rn(qf.x, (double)gp.x), dy = __dsub_rn(qf.y, (double)gp.y);
                key = __dadd_rn(ds.gen_cost[g], __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy))));
            }
        }
    }
    int best = key < INFINITY ? g : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ok = __shfl_xor_sync(0xffffffffu, key, o);
        const int og = __shfl_xor_sync(0xffffffffu, best, o);
        if (ok < key || (ok == key && og >= 0 && (best < 0 || og < best))) {
            key = ok;
            best = og;
        }
    }
    if (lane == 0) {
        *out_par = best;
        *out_dist = key;
    }
}

void launch_query_exact(const DevScene &ds, cudaStream_t st, const int32_t *field_parent, int i, int j, int qx,
                        int qy, double fx, double fy, int32_t *out_par, double *out_dist) {
    k_query_exact<<<1, 32, 0, st>>>(ds, field_parent, i, j, make_int2(qx, qy), make_double2(fx, fy), out_par,
                                    out_dist);
}

namespace {

// Lattice point inside the open interior of an obstacle?
__device__ bool centre_in_obstacle(const DevScene &ds, int px, int py) {
    const int bx = (px - ds.bin_x0) / ds.bin_size, by = (py - ds.bin_y0) / ds.bin_size;
    if (bx < 0 || by < 0 || bx >= ds.bin_nx || by >= ds.bin_ny) return false;
    const int bin = by * ds.bin_nx + bx;
    for (int it = ds.bin_start[bin]; it < ds.bin_start[bin + 1]; ++it) {
        const BinRec rec = ds.bin_recs[it];
        const int4 b4 = rec.box;
        if (px <= b4.x || px >= b4.z || py <= b4.y || py >= b4.w) continue;
        bool inside = true;
        for (int e = 0; e < rec.m && inside; ++e) {
            const int2 a = ds.poly_v[rec.voff + e], c = ds.poly_v[rec.voff + (e + 1 == rec.m ? 0 : e + 1)];
            inside = orient32(a.x, a.y, c.x, c.y, px, py) > 0;
        }
        if (inside) return true;
    }
    return false;
}

// Free-space mask of the pixel centres: bit (i % 32) of word j * free_words +
// i / 32 is set when pixel (i, j)'s centre lies outside the open interior of
// every obstacle. The obstacles are fixed for the scene's lifetime, so it is
// built once, one warp per word.
__global__ void k_free_mask(const __grid_constant__ DevScene ds, uint32_t *bits) {
    const long long w = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (w >= (long long)ds.Ny * ds.free_words) return;  // whole warps
    const int lane = threadIdx.x & 31;
    const int j = (int)(w / ds.free_words), i = (int)(w % ds.free_words) * 32 + lane;
    const int pitch_x = ds.S * ds.Wx / ds.Nx, pitch_y = ds.S * ds.Wy / ds.Ny;
    const bool is_free = i < ds.Nx && !centre_in_obstacle(ds, pitch_x * i + pitch_x / 2, pitch_y * j + pitch_y / 2);
    const unsigned m = __ballot_sync(0xffffffffu, is_free);
    if (lane == 0) bits[w] = m;
}

}  // namespace

void launch_free_mask(const DevScene &ds, cudaStream_t st, uint32_t *bits) {
    const long long words = (long long)ds.Ny * ds.free_words;
    const int per_block = NT / 32;
    k_free_mask<<<(unsigned)((words + per_block - 1) / per_block), NT, 0, st>>>(ds, bits);
}

void launch_pixel_phase(const DevScene &ds, cudaStream_t st, float *dist, int32_t *parent, int tile_row0,
                        int tile_row1) {
    const int tiles = ds.tiles_x * (tile_row1 - tile_row0);
    if (tiles <= 0) return;
    const int t0 = tile_row0 * ds.tiles_x;
    if (ds.use_maps && ds.gen_maps) {
        if (ds.tile == kTile) k_pixels<4, true><<<tiles, NT, 0, st>>>(ds, dist, parent, t0);
        else k_pixels<1, true><<<tiles, NT, 0, st>>>(ds, dist, parent, t0);
    } else {
        if (ds.tile == kTile) k_pixels<4, false><<<tiles, NT, 0, st>>>(ds, dist, parent, t0);
        else k_pixels<1, false><<<tiles, NT, 0, st>>>(ds, dist, parent, t0);
    }
}

void launch_pixel_phase_batched(const BatchDev &b, cudaStream_t st) {
    cudaMemsetAsync(b.tile_counter, 0, sizeof(int32_t), st);
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b.any_maps ? k_pixels_batched<true> : k_pixels_batched<false>,
                                                  NT, 0);
    const int grid = max(1, min(b.total_tiles, sms * max(per_sm, 1)));
    if (b.any_maps) k_pixels_batched<true><<<grid, NT, 0, st>>>(b);
    else k_pixels_batched<false><<<grid, NT, 0, st>>>(b);
}

int count_kernel_launches_pixel() { return 1; }

}  // namespace spm

#ifdef SPM_COUNT
// Instrumentation build only: reads and clears the work counters.
extern "C" int spm_debug_counters(unsigned long long *out32) {
    cudaDeviceSynchronize();
    if (cudaMemcpyFromSymbol(out32, spm::g_count, sizeof(unsigned long long) * 32) != cudaSuccess) return 1;
    unsigned long long z[32] = {0};
    cudaMemcpyToSymbol(spm::g_count, z, sizeof z);
    return 0;
}
#endif

#ifdef SPM_TIME
// Instrumentation build only: reads and clears the pixel kernel's phase clocks.
extern "C" int spm_debug_times(unsigned long long *out8) {
    cudaDeviceSynchronize();
    if (cudaMemcpyFromSymbol(out8, spm::g_time, sizeof(unsigned long long) * 8) != cudaSuccess) return 1;
    unsigned long long z[8] = {0};
    cudaMemcpyToSymbol(spm::g_time, z, sizeof z);
    return 0;
}
#endif
