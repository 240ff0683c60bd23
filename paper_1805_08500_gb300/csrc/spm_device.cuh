// spm_device.cuh -- exact geometric predicates used by the SPM kernels.
//
// All predicate inputs are points of the integer lattice whose span is at most
// 32767 units, so every coordinate difference fits in 16 signed bits, every
// product of two differences in 31 bits, and an orientation determinant
// (difference of two such products) in a signed 32-bit int: the int32
// arithmetic below is exact. Products that involve a squared segment length
// are done in int64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "spm_internal.h"

namespace spm {

// Work counters of an instrumentation build (-DSPM_COUNT); compiled out otherwise.
#ifdef SPM_COUNT
static __device__ unsigned long long g_count[32];  // one copy per translation unit
#define SPM_CNT(i, v) atomicAdd(&::spm::g_count[i], (unsigned long long)(v))
#define SPM_CNT_MAX(i, v) atomicMax(&::spm::g_count[i], (unsigned long long)(v))
#else
#define SPM_CNT(i, v) ((void)0)
#define SPM_CNT_MAX(i, v) ((void)0)
#endif

__device__ __forceinline__ int orient32(int ax, int ay, int bx, int by, int cx, int cy) {
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}
__device__ __forceinline__ int cross32(int ax, int ay, int bx, int by) { return ax * by - ay * bx; }

// Open segment p->q against the open interior of convex CCW polygon V[0..m).
// Separating-axis test on the segment and the polygon (both convex): they are
// disjoint in the interiors iff some outward edge normal of the polygon or the
// normal of the segment weakly separates them, i.e. (a) both endpoints lie on
// the closed outer side of one edge line, or (b) all polygon vertices lie on
// one closed side of the line pq. maskQ carries bit i = [orient(e_i, q) > 0].
__device__ __forceinline__ bool poly_blocks(const int2 *V, int m, int px, int py, int qx, int qy,
                                            unsigned maskQ) {
    unsigned mp = 0;
    int2 a = V[m - 1];
#pragma unroll 4
    for (int i = 0; i < m; ++i) {
        int2 b = V[i];
        // edge (a -> b) is edge index m-1 for i == 0, else i-1
        int e = (i == 0) ? m - 1 : i - 1;
        if (orient32(a.x, a.y, b.x, b.y, px, py) > 0) mp |= 1u << e;
        a = b;
    }
    if ((mp | maskQ) != ((1u << m) - 1u)) return false;
    const int dx = qx - px, dy = qy - py;
    bool pos = false, neg = false;
#pragma unroll 4
    for (int i = 0; i < m; ++i) {
        int s = dx * (V[i].y - py) - dy * (V[i].x - px);
        pos |= s > 0;
        neg |= s < 0;
    }
    return pos && neg;
}

__device__ __forceinline__ unsigned edge_mask(const int2 *V, int m, int qx, int qy) {
    unsigned mq = 0;
    for (int i = 0; i < m; ++i) {
        int2 a = V[i], b = V[i + 1 == m ? 0 : i + 1];
        if (orient32(a.x, a.y, b.x, b.y, qx, qy) > 0) mq |= 1u << i;
    }
    return mq;
}

// Same test with q = perpendicular foot of p on segment source A->B (Sec. 4),
// f = A + (num/den)(B - A), 0 < num < den. oA[i], oB[i] = orient(e_i, A / B).
// orient(e_i, f) has the sign of (den - num) * oA[i] + num * oB[i] (int64).
// The line p->f is parallel to perp(B - A) = (nx, ny).
__device__ __forceinline__ bool poly_blocks_foot(const int2 *V, int m, const int *oA,
                                                 const int *oB, int px, int py, long long num,
                                                 long long den, int nx, int ny) {
    unsigned mp = 0, mf = 0;
    for (int i = 0; i < m; ++i) {
        int2 a = V[i], b = V[i + 1 == m ? 0 : i + 1];
        if (orient32(a.x, a.y, b.x, b.y, px, py) > 0) mp |= 1u << i;
        long long of = (den - num) * (long long)oA[i] + num * (long long)oB[i];
        if (of > 0) mf |= 1u << i;
    }
    if ((mp | mf) != ((1u << m) - 1u)) return false;
    bool pos = false, neg = false;
    for (int i = 0; i < m; ++i) {
        int s = nx * (V[i].y - py) - ny * (V[i].x - px);
        pos |= s > 0;
        neg |= s < 0;
    }
    return pos && neg;
}

// Cone membership of direction w for a vertex generator: wedge cones are the
// closed CCW sector from c1 to c2 (angle < pi); ray cones the closed ray c1.
__device__ __forceinline__ bool in_cone(int ctype, int4 c, int wx, int wy) {
    if (ctype == kConeNone) return true;
    if (ctype == kConeWedge) return cross32(c.x, c.y, wx, wy) >= 0 && cross32(wx, wy, c.z, c.w) >= 0;
    if (ctype == kConeRay) return cross32(c.x, c.y, wx, wy) == 0 && c.x * wx + c.y * wy >= 0;
    return false;
}

// Shadow cone of vertex generator v with obstacle wedge (ws, we) (CCW) when
// reached along arrival direction d: the path wraps around the obstacle, so
// departures lie between d and the first wedge edge met when rotating from d
// toward the obstacle; empty when d points into the wedge.
__device__ __forceinline__ int make_cone(int4 wedge, int dx, int dy, int4 &c) {
    int a = cross32(dx, dy, wedge.x, wedge.y), b = cross32(dx, dy, wedge.z, wedge.w);
    if (a >= 0 && b >= 0 && (a | b)) {  // wedge on the left: turn counter-clockwise
        if (a == 0) { c = make_int4(dx, dy, dx, dy); return kConeRay; }
        c = make_int4(dx, dy, wedge.x, wedge.y);
        return kConeWedge;
    }
    if (a <= 0 && b <= 0 && (a | b)) {  // wedge on the right: turn clockwise
        if (b == 0) { c = make_int4(dx, dy, dx, dy); return kConeRay; }
        c = make_int4(wedge.z, wedge.w, dx, dy);
        return kConeWedge;
    }
    c = make_int4(0, 0, 0, 0);
    return kConeEmpty;
}

// in_cone(make_cone(wedge, d), w) written without branches (selects only):
// the same closed sector, ray or empty set. For tight loops where divergent
// branches cost more than the arithmetic.
__device__ __forceinline__ bool in_shadow_cone(int dx, int dy, short4 wedge, int wx, int wy) {
    const int a = cross32(dx, dy, wedge.x, wedge.y), b = cross32(dx, dy, wedge.z, wedge.w);
    const bool nz = (a | b) != 0;
    const bool left = (a >= 0) & (b >= 0) & nz, right = (a <= 0) & (b <= 0) & nz;
    const int cdw = cross32(dx, dy, wx, wy), dot = dx * wx + dy * wy;
    const bool ray_in = (cdw == 0) & (dot >= 0);
    const bool left_in = (cdw >= 0) & (cross32(wx, wy, wedge.x, wedge.y) >= 0);   // from d to the wedge start
    const bool right_in = (cdw <= 0) & (cross32(wedge.z, wedge.w, wx, wy) >= 0);  // from the wedge end to d
    return (left & ((a == 0) ? ray_in : left_in)) | (right & ((b == 0) ? ray_in : right_in));
}

// Arrival direction at generator v whose parent is u (lattice).
__device__ __forceinline__ void arrival_dir(const DevScene &ds, int u, int2 vl, int &dx, int &dy) {
    if (ds.gen_kind[u] == kSegI) {
        int4 L = ds.seg_lat[ds.gen_aux[u]];
        int ux = L.z - L.x, uy = L.w - L.y;
        int side = cross32(ux, uy, vl.x - L.x, vl.y - L.y);
        dx = side > 0 ? -uy : uy;
        dy = side > 0 ? ux : -ux;
        return;
    }
    int2 ul = ds.gen_lat[u];
    dx = vl.x - ul.x;
    dy = vl.y - ul.y;
}

// Conservative bin enumeration for the segment p->q thickened by r (lattice
// units, float). Calls f(bin) for every bin the thick segment may touch, in
// columns ordered from p toward q; stops early when f returns true.
template <class F>
__device__ __forceinline__ bool walk_bins(const DevScene &ds, float px, float py, float qx, float qy,
                                          float r, F &&f) {
    const float bs = (float)ds.bin_size, x0 = (float)ds.bin_x0, y0 = (float)ds.bin_y0;
    const float m = r + 1.0f;
    auto bin_of = [&](float v, float o, int n) {
        int b = (int)floorf((v - o) / bs);
        return b < 0 ? 0 : (b >= n ? n - 1 : b);
    };
    const int c0 = bin_of(fminf(px, qx) - m, x0, ds.bin_nx), c1 = bin_of(fmaxf(px, qx) + m, x0, ds.bin_nx);
    const float dx = qx - px, dy = qy - py;
    const int step = dx >= 0.f ? 1 : -1;
    const int cs = step > 0 ? c0 : c1, ce = step > 0 ? c1 : c0;
    for (int c = cs;; c += step) {
        float ylo, yhi;
        if (fabsf(dx) < 0.5f) {
            ylo = fminf(py, qy);
            yhi = fmaxf(py, qy);
        } else {
            float a = x0 + c * bs - m, b = x0 + (c + 1) * bs + m;
            float t0 = (a - px) / dx, t1 = (b - px) / dx;
            float tl = fmaxf(0.f, fminf(t0, t1)), th = fminf(1.f, fmaxf(t0, t1));
            if (tl > th) { tl = 0.f; th = 1.f; }  // rounding guard: keep it conservative
            float ya = py + tl * dy, yb = py + th * dy;
            ylo = fminf(ya, yb);
            yhi = fmaxf(ya, yb);
        }
        int r0 = bin_of(ylo - m, y0, ds.bin_ny), r1 = bin_of(yhi + m, y0, ds.bin_ny);
        int rstep = dy >= 0.f ? 1 : -1;
        int rs = rstep > 0 ? r0 : r1, re = rstep > 0 ? r1 : r0;
        for (int rr = rs;; rr += rstep) {
            if (f(rr * ds.bin_nx + c)) return true;
            if (rr == re) break;
        }
        if (c == ce) break;
    }
    return false;
}

// Does the (float, lattice units) segment p->q come within r of box [x0,x1]x[y0,y1]?
// Slab test on the box grown by r + 1: conservative (the 1e-4 slack on the
// segment parameter is far above the error of the fast divisions).
__device__ __forceinline__ bool seg_near_box(float px, float py, float qx, float qy, float r, int4 box) {
    const float m = r + 1.0f;
    float lo = 0.f, hi = 1.f;
    float d[2] = {qx - px, qy - py}, p[2] = {px, py};
    float bl[2] = {(float)box.x - m, (float)box.y - m}, bh[2] = {(float)box.z + m, (float)box.w + m};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (fabsf(d[k]) < 1e-6f) {
            if (p[k] < bl[k] || p[k] > bh[k]) return false;
        } else {
            const float id = __fdividef(1.0f, d[k]);
            float t0 = (bl[k] - p[k]) * id, t1 = (bh[k] - p[k]) * id;
            lo = fmaxf(lo, fminf(t0, t1));
            hi = fminf(hi, fmaxf(t0, t1));
        }
    }
    return lo <= hi + 1e-4f;
}

// Exact visibility between lattice point p and generator target q (a point),
// one thread: walks the bins along the segment and tests every polygon there.
__device__ __forceinline__ bool visible_points(const DevScene &ds, int px, int py, int qx, int qy) {
    if (px == qx && py == qy) return true;
    int4 sb = make_int4(min(px, qx), min(py, qy), max(px, qx), max(py, qy));
    bool blocked = walk_bins(ds, (float)px, (float)py, (float)qx, (float)qy, 0.f, [&](int bin) {
        SPM_CNT(24, 1);  // a bin walked
        for (int it = ds.bin_start[bin]; it < ds.bin_start[bin + 1]; ++it) {
            const BinRec rec = ds.bin_recs[it];
            const int4 bx = rec.box;
            if (bx.z < sb.x || bx.x > sb.z || bx.w < sb.y || bx.y > sb.w) continue;
            SPM_CNT(25, 1);  // a polygon tested
            const int2 *V = ds.poly_v + rec.voff;
            if (poly_blocks(V, rec.m, px, py, qx, qy, edge_mask(V, rec.m, qx, qy))) return true;
        }
        return false;
    });
    return !blocked;
}

// Exact visibility between lattice point p and its perpendicular foot on
// segment source s (0 < num < den), one thread. The bins are walked from p,
// or from the foot (from_foot); the result is the same (each bin's test is
// the whole segment's, and the walks cover every bin the segment crosses).
__device__ __forceinline__ bool visible_foot(const DevScene &ds, int s, int px, int py, long long num,
                                             long long den, bool from_foot = false) {
    int4 L = ds.seg_lat[s];
    int ux = L.z - L.x, uy = L.w - L.y;
    int side = cross32(ux, uy, px - L.x, py - L.y);
    if (side == 0) return true;
    double t = (double)num / (double)den;
    float fx = (float)(L.x + t * ux), fy = (float)(L.y + t * uy);
    int4 sb = make_int4((int)floorf(fminf((float)px, fx)) - 1, (int)floorf(fminf((float)py, fy)) - 1,
                        (int)ceilf(fmaxf((float)px, fx)) + 1, (int)ceilf(fmaxf((float)py, fy)) + 1);
    const int nx = -uy, ny = ux;
    const float wx0 = from_foot ? fx : (float)px, wy0 = from_foot ? fy : (float)py;
    const float wx1 = from_foot ? (float)px : fx, wy1 = from_foot ? (float)py : fy;
    bool blocked = walk_bins(ds, wx0, wy0, wx1, wy1, 0.f, [&](int bin) {
        for (int it = ds.bin_start[bin]; it < ds.bin_start[bin + 1]; ++it) {
            const BinRec rec = ds.bin_recs[it];
            const int4 bx = rec.box;
            if (bx.z < sb.x || bx.x > sb.z || bx.w < sb.y || bx.y > sb.w) continue;
            const int m = rec.m;
            const int2 *V = ds.poly_v + rec.voff;
            int oA[kMaxPolyVerts], oB[kMaxPolyVerts];
            for (int i = 0; i < m; ++i) {
                int2 a = V[i], bb = V[i + 1 == m ? 0 : i + 1];
                oA[i] = orient32(a.x, a.y, bb.x, bb.y, L.x, L.y);
                oB[i] = orient32(a.x, a.y, bb.x, bb.y, L.z, L.w);
            }
            if (poly_blocks_foot(V, m, oA, oB, px, py, num, den, nx, ny)) return true;
        }
        return false;
    });
    return !blocked;
}

// Pseudo-angle of direction (x, y) != 0: monotone in the true angle, [0, 4),
// opposite directions differ by exactly 2. The angular depth maps of the
// flood and the pixel pass bin directions by it (kAngBins bins of width
// kAngW; kAngEps covers its float error, about 1e-6).
constexpr float kAngW = 4.0f / kAngBins;
constexpr float kAngEps = 1e-4f;
__device__ __forceinline__ float pang(float x, float y) {
    const float r = __fdividef(fabsf(y), fabsf(x) + fabsf(y));
    if (y >= 0.f) return x >= 0.f ? r : 2.f - r;
    return x < 0.f ? 2.f + r : 4.f - r;
}

// Exclusive prefix sum of one value per thread over a CTA of blockDim.x
// threads (a multiple of 32, at most 1024); every thread must call it.
// wsum: 32 shared slots. Returns the sum of the values of lower threads.
__device__ __forceinline__ long long cta_exclusive_scan(long long x, long long *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const long long w = lane < nwarp ? wsum[lane] : 0;
        long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nwarp) wsum[lane] = wi - w;
    }
    __syncthreads();
    const long long r = wsum[warp] + inc - x;
    __syncthreads();  // wsum may be reused right after
    return r;
}


// Phase clocks of an instrumentation build (-DSPM_TIME); compiled out otherwise.
#ifdef SPM_TIME
// phase clocks of thread 0 (CTA wall time, barriers included), kept in
// registers and added to the global totals once at the end
static __device__ unsigned long long g_time[8];
#define SPM_T0()                                 \
    long long spm_t_ = clock64();                \
    unsigned long long spm_acc_[8] = {0, 0, 0, 0, 0, 0, 0, 0}
#define SPM_LAP(i)                                              \
    do {                                                        \
        const long long n_ = clock64();                         \
        spm_acc_[i] += (unsigned long long)(n_ - spm_t_);       \
        spm_t_ = n_;                                            \
    } while (0)
#define SPM_TFLUSH()                                                          \
    do {                                                                      \
        if (threadIdx.x == 0)                                                 \
            for (int i_ = 0; i_ < 8; ++i_) atomicAdd(&::spm::g_time[i_], spm_acc_[i_]); \
    } while (0)
#else
#define SPM_T0() ((void)0)
#define SPM_LAP(i) ((void)0)
#define SPM_TFLUSH() ((void)0)
#endif

// True when one polygon hides every point of the box from the point
// generator at lattice point g. The set of points whose open segment to g
// meets a convex polygon's interior is convex, so it suffices that the four
// corners of the pixel-centre box are hidden by the same polygon. Walks the
// bins of the thick segment (tile centre -> g, radius r) from the tile side
// and stops at the first such polygon.
__device__ __forceinline__ bool box_hidden(const DevScene &ds, int2 g, int4 box, float cx, float cy, float r,
                                           float max_len = 3.4e38f) {
    // walk toward g, optionally only the first max_len units (any subset of
    // polygons keeps the test exact)
    float tx = (float)g.x, ty = (float)g.y;
    const float dx = tx - cx, dy = ty - cy, len = sqrtf(dx * dx + dy * dy);
    if (len > max_len) {
        tx = cx + dx * (max_len / len);
        ty = cy + dy * (max_len / len);
    }
    return walk_bins(ds, cx, cy, tx, ty, r, [&](int bin) {
        for (int it = ds.bin_start[bin]; it < ds.bin_start[bin + 1]; ++it) {
            const BinRec rec = ds.bin_recs[it];
            if (!seg_near_box(cx, cy, tx, ty, r, rec.box)) continue;
            const int m = rec.m;
            const int2 *V = ds.poly_v + rec.voff;
            const unsigned mg = edge_mask(V, m, g.x, g.y);
            if (poly_blocks(V, m, box.x, box.y, g.x, g.y, mg) && poly_blocks(V, m, box.z, box.y, g.x, g.y, mg) &&
                poly_blocks(V, m, box.x, box.w, g.x, g.y, mg) && poly_blocks(V, m, box.z, box.w, g.x, g.y, mg))
                return true;
        }
        return false;
    });
}

// Warp-cooperative form of box_hidden (every lane must call it with the same
// arguments): the thick segment from the box centre to g is cut into strips
// one bin wide along its major axis; lane l takes strips l, l + 32, ...
// (nearest the box first) and the warp stops at the first round in which
// some lane found a polygon hiding all four corners.
__device__ __forceinline__ bool box_hidden_warp(const DevScene &ds, int2 g, int4 box, float cx, float cy,
                                                float r) {
    const int lane = threadIdx.x & 31;
    const float tx = (float)g.x, ty = (float)g.y;
    const float bs = (float)ds.bin_size, m = r + 1.0f;
    const bool xmaj = fabsf(tx - cx) >= fabsf(ty - cy);
    // major axis: u (bins along it), minor: w
    const float pu = xmaj ? cx : cy, pw = xmaj ? cy : cx, qu = xmaj ? tx : ty, qw = xmaj ? ty : tx;
    const float ou = xmaj ? (float)ds.bin_x0 : (float)ds.bin_y0, ow = xmaj ? (float)ds.bin_y0 : (float)ds.bin_x0;
    const int nu = xmaj ? ds.bin_nx : ds.bin_ny, nw = xmaj ? ds.bin_ny : ds.bin_nx;
    auto bin_of = [&](float v, float o, int n) {
        int b = (int)floorf((v - o) / bs);
        return b < 0 ? 0 : (b >= n ? n - 1 : b);
    };
    const int u0 = bin_of(fminf(pu, qu) - m, ou, nu), u1 = bin_of(fmaxf(pu, qu) + m, ou, nu);
    const int ustep = qu >= pu ? 1 : -1, us = ustep > 0 ? u0 : u1;
    const int nstrips = u1 - u0 + 1;
    const float du = qu - pu, dw = qw - pw;
    for (int base = 0; base < nstrips; base += 32) {
        bool found = false;
        const int sidx = base + lane;
        if (sidx < nstrips) {
            const int u = us + ustep * sidx;
            float wlo, whi;
            if (fabsf(du) < 0.5f) {
                wlo = fminf(pw, qw);
                whi = fmaxf(pw, qw);
            } else {
                const float a = ou + u * bs - m, b = ou + (u + 1) * bs + m;
                const float t0 = (a - pu) / du, t1 = (b - pu) / du;
                float tl = fmaxf(0.f, fminf(t0, t1)), th = fminf(1.f, fmaxf(t0, t1));
                if (tl > th) { tl = 0.f; th = 1.f; }
                const float wa = pw + tl * dw, wb = pw + th * dw;
                wlo = fminf(wa, wb);
                whi = fmaxf(wa, wb);
            }
            const int w0 = bin_of(wlo - m, ow, nw), w1 = bin_of(whi + m, ow, nw);
            for (int w = w0; w <= w1 && !found; ++w) {
                const int bin = xmaj ? w * ds.bin_nx + u : u * ds.bin_nx + w;
                for (int it = ds.bin_start[bin]; it < ds.bin_start[bin + 1] && !found; ++it) {
                    const BinRec rec = ds.bin_recs[it];
                    if (!seg_near_box(cx, cy, tx, ty, r, rec.box)) continue;
                    const int2 *V = ds.poly_v + rec.voff;
                    const unsigned mg = edge_mask(V, rec.m, g.x, g.y);
                    found = poly_blocks(V, rec.m, box.x, box.y, g.x, g.y, mg) &&
                            poly_blocks(V, rec.m, box.z, box.y, g.x, g.y, mg) &&
                            poly_blocks(V, rec.m, box.x, box.w, g.x, g.y, mg) &&
                            poly_blocks(V, rec.m, box.z, box.w, g.x, g.y, mg);
                }
            }
        }
        if (__any_sync(0xffffffffu, found)) return true;
    }
    return false;
}

}  // namespace spm
