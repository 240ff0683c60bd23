// spm_prep.cpp -- host preparation of a shortest-path-map scene.
//
// Builds the generator table of arxiv 1805.08500 Sec. 3.1 (the DataArray:
// sources, then obstacle vertices) and Sec. 4 (each segment source adds its two
// endpoints plus one interior entry), snaps coordinates to the exact integer
// lattice, validates the geometry and bins polygons for the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <unordered_map>

#include <cuda_runtime.h>

#include "spm_internal.h"

namespace spm {
namespace {

using i64 = long long;

inline i64 orient(i64 ax, i64 ay, i64 bx, i64 by, i64 cx, i64 cy) {
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}
inline i64 cross(i64 ax, i64 ay, i64 bx, i64 by) { return ax * by - ay * bx; }

// Pseudo-angle order of integer directions starting at +x, counter-clockwise.
inline int upper(i64 x, i64 y) { return (y > 0 || (y == 0 && x > 0)) ? 0 : 1; }
inline bool ang_less(i64 ax, i64 ay, i64 bx, i64 by) {
    int ha = upper(ax, ay), hb = upper(bx, by);
    if (ha != hb) return ha < hb;
    return cross(ax, ay, bx, by) > 0;
}
// CCW angle from a to b is strictly less than pi?
inline bool ccw_less_than_pi(i64 ax, i64 ay, i64 bx, i64 by) { return cross(ax, ay, bx, by) > 0; }
// direction x inside closed CCW sector [s, e] of angle <= pi
inline bool in_closed_sector(i64 sx, i64 sy, i64 ex, i64 ey, i64 x, i64 y) {
    i64 se = cross(sx, sy, ex, ey);
    if (se == 0) return cross(sx, sy, x, y) >= 0;  // half-plane
    return cross(sx, sy, x, y) >= 0 && cross(x, y, ex, ey) >= 0;
}

struct Sector { i64 sx, sy, ex, ey; };

// Union of closed sectors around a point. Returns 1 and the arc when the
// union is one arc of angle < pi (a convex corner of free space), 0 when it
// is connected but not such an arc, -1 when it is disconnected (a pinch).
int union_arc(const std::vector<Sector> &secs, Sector &arc) {
    const int m = (int)secs.size();
    // an arc start is a sector start not covered by any other sector
    std::vector<int> starts;
    for (int a = 0; a < m; ++a) {
        bool covered = false;
        for (int k = 0; k < m && !covered; ++k) {
            if (k == a) continue;
            const Sector &s = secs[k];
            // start of a strictly inside sector k or equal to k's start with k wider
            if (in_closed_sector(s.sx, s.sy, s.ex, s.ey, secs[a].sx, secs[a].sy) &&
                !(cross(s.sx, s.sy, secs[a].sx, secs[a].sy) == 0 &&
                  s.sx * secs[a].sx + s.sy * secs[a].sy > 0 && k > a))
                covered = true;
        }
        if (!covered) starts.push_back(a);
    }
    if (starts.empty()) return 0;          // every start covered: full circle
    if (starts.size() > 1) return -1;      // several arcs: disconnected
    const Sector &s0 = secs[starts[0]];
    // grow the arc end: repeatedly absorb sectors whose start lies in the arc
    i64 ex = s0.ex, ey = s0.ey;
    std::vector<char> used(m, 0);
    used[starts[0]] = 1;
    for (bool grew = true; grew;) {
        grew = false;
        for (int k = 0; k < m; ++k) {
            if (used[k]) continue;
            // start of k inside [s0.start, end]: compare CCW angles from s0.start
            i64 rx = s0.sx, ry = s0.sy;
            auto rel = [&](i64 x, i64 y) {  // 0: [0, pi), 1: [pi, 2pi)
                i64 c = cross(rx, ry, x, y);
                return (c > 0 || (c == 0 && rx * x + ry * y > 0)) ? 0 : 1;
            };
            auto le = [&](i64 ax, i64 ay, i64 bx, i64 by) {  // rel angle a <= rel angle b
                int ha = rel(ax, ay), hb = rel(bx, by);
                if (ha != hb) return ha < hb;
                return cross(ax, ay, bx, by) >= 0;
            };
            if (le(secs[k].sx, secs[k].sy, ex, ey)) {
                used[k] = 1;
                grew = true;
                if (!le(secs[k].ex, secs[k].ey, ex, ey)) { ex = secs[k].ex; ey = secs[k].ey; }
            }
        }
    }
    if (!ccw_less_than_pi(s0.sx, s0.sy, ex, ey)) return 0;
    arc = {s0.sx, s0.sy, ex, ey};
    return 1;
}

bool closed_polygon_contains(const HostScene &hs, int k, i64 x, i64 y) {
    int b = hs.poly_off[k], m = hs.poly_off[k + 1] - b;
    for (int i = 0; i < m; ++i) {
        int j = (i + 1) % m;
        if (orient(hs.poly_v[2 * (b + i)], hs.poly_v[2 * (b + i) + 1], hs.poly_v[2 * (b + j)],
                   hs.poly_v[2 * (b + j) + 1], x, y) < 0)
            return false;
    }
    return true;
}

template <class F>
void for_polys_near(const HostScene &hs, i64 x0, i64 y0, i64 x1, i64 y1, F &&f) {
    auto bx = [&](i64 x) { return (int)std::max<i64>(0, std::min<i64>(hs.bin_nx - 1, (x - hs.bin_x0) / hs.bin_size)); };
    auto by = [&](i64 y) { return (int)std::max<i64>(0, std::min<i64>(hs.bin_ny - 1, (y - hs.bin_y0) / hs.bin_size)); };
    int cx0 = bx(x0), cx1 = bx(x1), cy0 = by(y0), cy1 = by(y1);
    std::vector<int> seen;
    for (int cy = cy0; cy <= cy1; ++cy)
        for (int cx = cx0; cx <= cx1; ++cx) {
            int c = cy * hs.bin_nx + cx;
            for (int it = hs.bin_start[c]; it < hs.bin_start[c + 1]; ++it) {
                int k = hs.bin_items[it];
                if (std::find(seen.begin(), seen.end(), k) != seen.end()) continue;
                seen.push_back(k);
                f(k);
            }
        }
}

spm_status fail(std::string &err, spm_status st, const char *msg) {
    err = msg;
    return st;
}

// A source point must lie inside the world and outside every closed obstacle.
spm_status check_free(const HostScene &hs, i64 x, i64 y, std::string &err, const char *what) {
    if (x < 0 || y < 0 || x > (i64)hs.Wx * hs.S || y > (i64)hs.Wy * hs.S) {
        err = std::string(what) + " outside the world";
        return SPM_ERR_BAD_GEOMETRY;
    }
    bool bad = false;
    for_polys_near(hs, x, y, x, y, [&](int k) { bad |= closed_polygon_contains(hs, k, x, y); });
    if (bad) {
        err = std::string(what) + " is not strictly outside every obstacle";
        return SPM_ERR_BAD_GEOMETRY;
    }
    return SPM_OK;
}

// Closed segment and closed convex polygon disjoint? (strict separating axis)
bool segment_clear_of_poly(const HostScene &hs, int k, i64 ax, i64 ay, i64 bx, i64 by) {
    int b = hs.poly_off[k], m = hs.poly_off[k + 1] - b;
    const int32_t *V = hs.poly_v.data() + 2 * b;
    for (int i = 0; i < m; ++i) {
        int j = (i + 1) % m;
        if (orient(V[2 * i], V[2 * i + 1], V[2 * j], V[2 * j + 1], ax, ay) < 0 &&
            orient(V[2 * i], V[2 * i + 1], V[2 * j], V[2 * j + 1], bx, by) < 0)
            return true;
    }
    bool pos = false, neg = false, zero = false;
    for (int i = 0; i < m; ++i) {
        i64 o = orient(ax, ay, bx, by, V[2 * i], V[2 * i + 1]);
        pos |= o > 0;
        neg |= o < 0;
        zero |= o == 0;
    }
    return !zero && !(pos && neg);
}

spm_status snap_sources(HostScene &hs, const float *pts, const float *segs, std::string &err) {
    const int np = (int)hs.points.size() / 2, ns = (int)hs.segs.size() / 4;
    for (int i = 0; i < 2 * np; ++i) hs.points[i] = pts[i];
    for (int i = 0; i < 4 * ns; ++i) hs.segs[i] = segs[i];
    for (float v : hs.points)
        if (!std::isfinite(v)) return fail(err, SPM_ERR_BAD_GEOMETRY, "non-finite point source");
    for (float v : hs.segs)
        if (!std::isfinite(v)) return fail(err, SPM_ERR_BAD_GEOMETRY, "non-finite segment source");
    for (float v : hs.points)
        if (std::fabs(std::nearbyint((double)v * (double)hs.S)) > 1073741824.0)
            return fail(err, SPM_ERR_BAD_GEOMETRY, "point source outside the world");
    for (float v : hs.segs)
        if (std::fabs(std::nearbyint((double)v * (double)hs.S)) > 1073741824.0)
            return fail(err, SPM_ERR_BAD_GEOMETRY, "segment endpoint outside the world");
    auto snap = [&](float v) { return (int32_t)std::nearbyint((double)v * (double)hs.S); };
    int g = 0;
    for (int i = 0; i < np; ++i, ++g) {
        int32_t x = snap(hs.points[2 * i]), y = snap(hs.points[2 * i + 1]);
        spm_status st = check_free(hs, x, y, err, "point source");
        if (st != SPM_OK) return st;
        hs.gen_lat[2 * g] = x;
        hs.gen_lat[2 * g + 1] = y;
        hs.gen_pos[2 * g] = hs.points[2 * i];
        hs.gen_pos[2 * g + 1] = hs.points[2 * i + 1];
    }
    for (int s = 0; s < ns; ++s) {
        int32_t L[4];
        for (int c = 0; c < 4; ++c) L[c] = snap(hs.segs[4 * s + c]);
        if (L[0] == L[2] && L[1] == L[3]) return fail(err, SPM_ERR_BAD_GEOMETRY, "zero-length segment source");
        spm_status st = check_free(hs, L[0], L[1], err, "segment endpoint");
        if (st == SPM_OK) st = check_free(hs, L[2], L[3], err, "segment endpoint");
        if (st != SPM_OK) return st;
        bool touch = false;
        for_polys_near(hs, std::min(L[0], L[2]), std::min(L[1], L[3]), std::max(L[0], L[2]),
                       std::max(L[1], L[3]),
                       [&](int k) { touch |= !segment_clear_of_poly(hs, k, L[0], L[1], L[2], L[3]); });
        if (touch) return fail(err, SPM_ERR_BAD_GEOMETRY, "segment source touches an obstacle");
        for (int c = 0; c < 4; ++c) hs.seg_lat[4 * s + c] = L[c];
        for (int c = 0; c < 3; ++c, ++g) {
            int o = (c == 1) ? 2 : 0;  // A, B, interior (stored at A)
            hs.gen_lat[2 * g] = L[o];
            hs.gen_lat[2 * g + 1] = L[o + 1];
            hs.gen_pos[2 * g] = hs.segs[4 * s + o];
            hs.gen_pos[2 * g + 1] = hs.segs[4 * s + o + 1];
        }
    }
    return SPM_OK;
}

}  // namespace

spm_status prepare_scene(const spm_scene_desc &d, HostScene &hs, std::string &err) {
    if (d.world_w <= 0 || d.world_h <= 0 || d.grid_w <= 0 || d.grid_h <= 0)
        return fail(err, SPM_ERR_INVALID_ARG, "world and grid sizes must be positive");
    if (d.n_polys < 0 || d.n_points < 0 || d.n_segments < 0)
        return fail(err, SPM_ERR_INVALID_ARG, "negative count");
    if (d.n_points + d.n_segments < 1) return fail(err, SPM_ERR_INVALID_ARG, "scene has no source");
    if ((d.n_polys > 0 && (!d.poly_offsets || !d.poly_xy)) || (d.n_points > 0 && !d.point_xy) ||
        (d.n_segments > 0 && !d.seg_xyxy))
        return fail(err, SPM_ERR_INVALID_ARG, "null array for a non-zero count");
    if ((int64_t)d.grid_w * d.grid_h > (int64_t)1 << 31)
        return fail(err, SPM_ERR_INVALID_ARG, "grid too large");
    hs.Wx = d.world_w; hs.Wy = d.world_h; hs.Nx = d.grid_w; hs.Ny = d.grid_h;
    const int P = d.n_polys;
    if (P > 0 && d.poly_offsets[0] != 0) return fail(err, SPM_ERR_INVALID_ARG, "poly_offsets[0] != 0");
    for (int k = 0; k < P; ++k)
        if (d.poly_offsets[k + 1] - d.poly_offsets[k] < 3 ||
            d.poly_offsets[k + 1] - d.poly_offsets[k] > kMaxPolyVerts)
            return fail(err, SPM_ERR_BAD_GEOMETRY, "polygon must have 3..16 vertices");
    const int V = P ? d.poly_offsets[P] : 0;
    // lattice scale: pixel centres on the lattice, span within 15 bits
    i64 S = 1;
    while (((S * d.world_w) % (2 * (i64)d.grid_w)) || ((S * d.world_h) % (2 * (i64)d.grid_h))) {
        S *= 2;
        if (S > 32768) return fail(err, SPM_ERR_BAD_GEOMETRY, "pixel centres are not on a power-of-two lattice");
    }
    i64 lo_x = 0, lo_y = 0, hi_x = d.world_w, hi_y = d.world_h;
    for (int i = 0; i < V; ++i) {
        lo_x = std::min<i64>(lo_x, d.poly_xy[2 * i]);
        hi_x = std::max<i64>(hi_x, d.poly_xy[2 * i]);
        lo_y = std::min<i64>(lo_y, d.poly_xy[2 * i + 1]);
        hi_y = std::max<i64>(hi_y, d.poly_xy[2 * i + 1]);
    }
    const i64 span = std::max(hi_x - lo_x, hi_y - lo_y);
    if (S * span > 32767) return fail(err, SPM_ERR_BAD_GEOMETRY, "scene span too large for the exact 15-bit lattice");
    while (2 * S * span <= 32767) S *= 2;
    hs.S = (int32_t)S;
    // polygons: lattice, counter-clockwise, strictly convex
    hs.poly_off.assign(P + 1, 0);
    hs.poly_v.assign(2 * V, 0);
    hs.poly_box.assign(4 * P, 0);
    for (int k = 0; k < P; ++k) {
        int b = d.poly_offsets[k], m = d.poly_offsets[k + 1] - b;
        i64 area2 = 0;
        for (int i = 0; i < m; ++i) {
            int j = (i + 1) % m;
            area2 += (i64)d.poly_xy[2 * (b + i)] * d.poly_xy[2 * (b + j) + 1] -
                     (i64)d.poly_xy[2 * (b + j)] * d.poly_xy[2 * (b + i) + 1];
        }
        if (area2 == 0) return fail(err, SPM_ERR_BAD_GEOMETRY, "degenerate polygon");
        for (int i = 0; i < m; ++i) {
            int src = area2 > 0 ? b + i : b + (m - 1 - i);
            hs.poly_v[2 * (b + i)] = (int32_t)(d.poly_xy[2 * src] * S);
            hs.poly_v[2 * (b + i) + 1] = (int32_t)(d.poly_xy[2 * src + 1] * S);
        }
        hs.poly_off[k + 1] = b + m;
        i64 x0 = hs.poly_v[2 * b], x1 = x0, y0 = hs.poly_v[2 * b + 1], y1 = y0;
        for (int i = 0; i < m; ++i) {
            const int32_t *a = &hs.poly_v[2 * (b + i)], *bb = &hs.poly_v[2 * (b + (i + 1) % m)],
                          *c = &hs.poly_v[2 * (b + (i + 2) % m)];
            if (orient(a[0], a[1], bb[0], bb[1], c[0], c[1]) <= 0)
                return fail(err, SPM_ERR_BAD_GEOMETRY, "polygon is not strictly convex");
            x0 = std::min<i64>(x0, a[0]); x1 = std::max<i64>(x1, a[0]);
            y0 = std::min<i64>(y0, a[1]); y1 = std::max<i64>(y1, a[1]);
        }
        hs.poly_box[4 * k] = (int32_t)x0; hs.poly_box[4 * k + 1] = (int32_t)y0;
        hs.poly_box[4 * k + 2] = (int32_t)x1; hs.poly_box[4 * k + 3] = (int32_t)y1;
    }
    // bins: about four per polygon, square, covering world and polygons
    {
        i64 bx0 = lo_x * S - 1, by0 = lo_y * S - 1, bx1 = hi_x * S + 1, by1 = hi_y * S + 1;
        double area = (double)(bx1 - bx0) * (double)(by1 - by0);
        i64 bs = (i64)std::ceil(std::sqrt(area / (4.0 * std::max(1, P))));
        bs = std::max<i64>(bs, 8);
        hs.bin_x0 = (int32_t)bx0; hs.bin_y0 = (int32_t)by0; hs.bin_size = (int32_t)bs;
        hs.bin_nx = (int32_t)((bx1 - bx0) / bs + 1);
        hs.bin_ny = (int32_t)((by1 - by0) / bs + 1);
        const int nb = hs.bin_nx * hs.bin_ny;
        hs.bin_start.assign(nb + 1, 0);
        std::vector<int32_t> fillc(nb, 0);
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
                for (int c = 0; c < nb; ++c) hs.bin_start[c + 1] += hs.bin_start[c];
                hs.bin_items.assign(hs.bin_start[nb], 0);
            }
            for (int k = 0; k < P; ++k) {
                int cx0 = (int)((hs.poly_box[4 * k] - bx0) / bs), cx1 = (int)((hs.poly_box[4 * k + 2] - bx0) / bs);
                int cy0 = (int)((hs.poly_box[4 * k + 1] - by0) / bs), cy1 = (int)((hs.poly_box[4 * k + 3] - by0) / bs);
                for (int cy = cy0; cy <= cy1; ++cy)
                    for (int cx = cx0; cx <= cx1; ++cx) {
                        int c = cy * hs.bin_nx + cx;
                        if (pass == 0) hs.bin_start[c + 1]++;
                        else hs.bin_items[hs.bin_start[c] + fillc[c]++] = k;
                    }
            }
        }
    }
    // sources
    const int npt = d.n_points, nseg = d.n_segments;
    hs.points.assign(2 * npt, 0.f);
    hs.segs.assign(4 * nseg, 0.f);
    hs.seg_lat.assign(4 * nseg, 0);
    hs.n_src = npt + 3 * nseg;
    hs.gen_kind.assign(hs.n_src, 0);
    hs.gen_aux.assign(hs.n_src, 0);
    hs.gen_lat.assign(2 * hs.n_src, 0);
    hs.gen_pos.assign(2 * hs.n_src, 0.f);
    hs.gen_wedge.assign(4 * hs.n_src, 0);
    for (int i = 0; i < npt; ++i) { hs.gen_kind[i] = kPoint; hs.gen_aux[i] = i; }
    for (int s = 0; s < nseg; ++s)
        for (int c = 0; c < 3; ++c) {
            hs.gen_kind[npt + 3 * s + c] = kSegA + c;
            hs.gen_aux[npt + 3 * s + c] = s;
        }
    spm_status st = snap_sources(hs, d.point_xy, d.seg_xyxy, err);
    if (st != SPM_OK) return st;
    // obstacle vertices that are convex corners of the union of obstacles
    std::unordered_map<i64, int> seen;
    seen.reserve(2 * V + 1);
    for (int k = 0; k < P; ++k) {
        const int b = hs.poly_off[k], m = hs.poly_off[k + 1] - b;
        for (int i = 0; i < m; ++i) {
            const i64 vx = hs.poly_v[2 * (b + i)], vy = hs.poly_v[2 * (b + i) + 1];
            const i64 key = (vx + (1 << 20)) * (1ll << 22) + (vy + (1 << 20));
            if (!seen.emplace(key, b + i).second) continue;  // later duplicates
            std::vector<Sector> secs;
            bool interior = false;
            for_polys_near(hs, vx, vy, vx, vy, [&](int q) {
                if (interior) return;
                const int qb = hs.poly_off[q], qm = hs.poly_off[q + 1] - qb;
                const int32_t *Q = hs.poly_v.data() + 2 * qb;
                int zeros = 0, ze = -1, vid = -1;
                for (int j = 0; j < qm; ++j) {
                    int jn = (j + 1) % qm;
                    i64 o = orient(Q[2 * j], Q[2 * j + 1], Q[2 * jn], Q[2 * jn + 1], vx, vy);
                    if (o < 0) return;  // outside q
                    if (o == 0) { ++zeros; ze = j; }
                    if (Q[2 * j] == vx && Q[2 * j + 1] == vy) vid = j;
                }
                if (zeros == 0) { interior = true; return; }
                if (vid >= 0) {
                    int nx = (vid + 1) % qm, pv = (vid + qm - 1) % qm;
                    secs.push_back({Q[2 * nx] - vx, Q[2 * nx + 1] - vy, Q[2 * pv] - vx, Q[2 * pv + 1] - vy});
                } else {
                    int jn = (ze + 1) % qm;
                    i64 ex = Q[2 * jn] - Q[2 * ze], ey = Q[2 * jn + 1] - Q[2 * ze + 1];
                    secs.push_back({ex, ey, -ex, -ey});
                }
            });
            if (interior) continue;
            Sector arc;
            int r = union_arc(secs, arc);
            if (r < 0) return fail(err, SPM_ERR_BAD_GEOMETRY, "obstacles touch at a single point");
            if (r == 0) continue;
            hs.gen_kind.push_back(kVert);
            hs.gen_aux.push_back(b + i);
            hs.gen_lat.push_back((int32_t)vx);
            hs.gen_lat.push_back((int32_t)vy);
            hs.gen_pos.push_back((float)(vx / S));
            hs.gen_pos.push_back((float)(vy / S));
            hs.gen_wedge.push_back((int32_t)arc.sx);
            hs.gen_wedge.push_back((int32_t)arc.sy);
            hs.gen_wedge.push_back((int32_t)arc.ex);
            hs.gen_wedge.push_back((int32_t)arc.ey);
        }
    }
    hs.n_gen = (int32_t)hs.gen_kind.size();
    hs.n_vert = hs.n_gen - hs.n_src;
    return SPM_OK;
}

spm_status update_sources(HostScene &hs, const float *pts, const float *segs, std::string &err) {
    const int np = (int)hs.points.size() / 2, ns = (int)hs.segs.size() / 4;
    if ((np > 0 && !pts) || (ns > 0 && !segs)) return fail(err, SPM_ERR_INVALID_ARG, "null source array");
    HostScene copy = hs;
    spm_status st = snap_sources(copy, pts, segs, err);
    if (st != SPM_OK) return st;
    hs = std::move(copy);
    return SPM_OK;
}

}  // namespace spm
