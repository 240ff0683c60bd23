/*
 * spm_oracle.c -- plain CPU FP64 reference for shortest-path maps (SPMs).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls
 * this file; only tests/, the smoke check and the benchmark's CPU-baseline /
 * reference leg do. It shares no code with the CUDA library.
 *
 * What it computes (arxiv 1805.08500, Sec. 3 "Multi-Source Shortest Path Maps"
 * and Sec. 4 "Segment Sources"):
 *   lambda*(p)  = length of the globally shortest obstacle-avoiding path from
 *                 pixel centre p to the closest point source or the closest
 *                 reachable point of the closest segment source (Sec. 3, Sec. 4);
 *   parent(p)   = the next point on that path, i.e. a source, a segment
 *                 endpoint / interior foot, or an obstacle vertex (Sec. 3.1,
 *                 the ParentId field of the DataArray).
 * Euclidean shortest paths among polygons bend only at obstacle vertices (the
 * visibility-graph theorem the paper cites in Sec. 1-2), so the oracle is the
 * plain definition written out:
 *   1. vertex costs by Dijkstra over the visibility graph among sources and
 *      obstacle vertices (the paper's Procedure 1 "Search" picks the minimum
 *      unexpanded entry, Procedure 4 "Distance" relaxes the visible ones);
 *   2. per pixel, the minimum over visible generators g of cost(g) + |p - g|
 *      (Procedure 3 "Cone", the strict-less depth test), taken in exact
 *      (key, id) order; segment interiors use the perpendicular foot (Sec. 4).
 * Visibility is exact: a segment is blocked iff its open interior meets the
 * open interior of some convex obstacle, decided by Cyrus-Beck parametric
 * clipping with rational comparisons in __int128.
 *
 * Readings of points the paper leaves open: pixel
 * sample = pixel centre (Sec. 6 discussion); touching or grazing obstacle
 * boundaries is allowed; vertex generators are restricted to their shadow
 * cone behind their parent; ties go to the smaller generator id.
 *
 * Coordinates for predicates are snapped to an integer lattice of scale S
 * (S a power of two, all pixel centres on the lattice, as fine as keeps every
 * coordinate within 2^24 lattice units), so every orientation determinant is
 * an exact integer in int64 and every comparison of two rational parameters
 * exact in __int128. Distances use the true (unsnapped) coordinates in FP64.
 * Obstacle vertices and pixel centres lie on the lattice exactly. Sources are
 * rounded to it: by default (snapping "pixel") to the coarser sub-lattice of
 * scale Sp, the largest power of two with every pixel centre on it and
 * Sp * span <= 32767 -- the predicate lattice the GPU library uses, whose
 * reading of a moved source's visibility this reproduces -- or (snapping
 * "fine") to the full lattice, which puts a source within 1 / (2 S) of where
 * it is. Exact predicates do not depend on the scale of the lattice, only on
 * the points, so both give the same result wherever the sources are
 * lattice points of both.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef long long ll;
typedef __int128 i128;

enum { K_POINT = 0, K_SEGA = 1, K_SEGB = 2, K_SEGI = 3, K_VERT = 4 };
enum { O_OK = 0, O_EARG = 1, O_EGEOM = 2, O_ENOMEM = 3 };
enum { CONE_NONE = 0, CONE_LEFT = 1, CONE_RIGHT = 2, CONE_EMPTY = 3 };

typedef struct {
    ll Wx, Wy;
    int Nx, Ny;
    ll S;      /* predicate lattice */
    ll Sp;     /* the coarser lattice "pixel" snapping rounds sources to (0: none, the scene is too wide) */
    int fine;  /* snap sources to the full lattice */
    /* polygons, lattice coordinates, counter-clockwise */
    int np;
    int *po;
    ll *px, *py;
    ll *bx0, *by0, *bx1, *by1;
    /* segment sources: true and lattice endpoints */
    int nseg;
    double *sf;  /* 4 per segment */
    ll *sl;      /* 4 per segment */
    /* generators */
    int ng, nsrc;
    int *kind, *sidx;
    double *tx, *ty;
    ll *lx, *ly;
    ll *wsx, *wsy, *wex, *wey; /* obstacle wedge of vertex generators (CCW) */
    double *cost;
    int *par;
    ll *cdx, *cdy; /* arrival direction at a vertex generator */
    int *cside;    /* CONE_* */
    /* uniform cell grid of polygon bounding boxes */
    ll gx0, gy0, gcs;
    int gnx, gny;
    int *gstart, *gitems;
    /* dense visibility bits: generator u (row) -> vertex generator v (column) */
    unsigned char *vis;
    int nvert, vbase;
    char err[256];
} orc_t;

static ll orient(ll ax, ll ay, ll bx, ll by, ll cx, ll cy) {
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}
static ll cross2(ll ax, ll ay, ll bx, ll by) { return ax * by - ay * bx; }
static int sgn(ll v) { return (v > 0) - (v < 0); }

/* ------------------------------------------------------------------------ */
/* exact segment-vs-convex-polygon test (Cyrus-Beck with rational bounds)   */
/* ------------------------------------------------------------------------ */

/* fraction n/d with d > 0 */
typedef struct { ll n, d; } frac_t;
static int frac_lt(frac_t a, frac_t b) { return (i128)a.n * b.d < (i128)b.n * a.d; }

/* Points X(u) = p + u*D, u in the open interval (0, U). Returns 1 iff some
 * such point lies in the open interior of polygon k (intersection of the open
 * left half-planes of its CCW edges). */
static int blocked_by_poly(const orc_t *o, int k, ll px, ll py, ll Dx, ll Dy, frac_t U) {
    frac_t lo = {0, 1}, hi = U;
    int b = o->po[k], e = o->po[k + 1], m = e - b;
    for (int i = 0; i < m; i++) {
        ll ax = o->px[b + i], ay = o->py[b + i];
        ll bx = o->px[b + (i + 1) % m], by = o->py[b + (i + 1) % m];
        ll c0 = orient(ax, ay, bx, by, px, py);       /* value at u = 0 */
        ll k1 = cross2(bx - ax, by - ay, Dx, Dy);     /* slope in u */
        if (k1 == 0) {
            if (c0 > 0) continue;
            return 0;
        }
        if (k1 > 0) { /* u > -c0/k1 */
            frac_t f = {-c0, k1};
            if (frac_lt(lo, f)) lo = f;
        } else { /* u < c0/(-k1) */
            frac_t f = {c0, -k1};
            if (frac_lt(f, hi)) hi = f;
        }
        if (!frac_lt(lo, hi)) return 0;
    }
    return frac_lt(lo, hi);
}

/* Visit polygons whose bounding box may meet the segment p -> p + U*D. The
 * segment is cut into pieces no longer than half a cell; each piece's box
 * (widened by one lattice unit) selects grid cells, so every polygon the
 * segment touches is visited. */
static int segment_blocked(const orc_t *o, ll px, ll py, ll Dx, ll Dy, frac_t U,
                           int *stamp, int *tick) {
    double u1 = (double)U.n / (double)U.d;
    double ex = (double)Dx * u1, ey = (double)Dy * u1;
    double len = sqrt(ex * ex + ey * ey);
    int pieces = (int)(len / (0.5 * (double)o->gcs)) + 1;
    (*tick)++;
    if (*tick == 0x7fffffff) {
        memset(stamp, 0, sizeof(int) * o->np);
        *tick = 1;
    }
    double sx0 = (double)px, sy0 = (double)py;
    ll qx_lo = 0, qx_hi = 0, qy_lo = 0, qy_hi = 0;
    {
        double fx = sx0 + ex, fy = sy0 + ey;
        qx_lo = (ll)floor(fmin(sx0, fx)) - 1; qx_hi = (ll)ceil(fmax(sx0, fx)) + 1;
        qy_lo = (ll)floor(fmin(sy0, fy)) - 1; qy_hi = (ll)ceil(fmax(sy0, fy)) + 1;
    }
    for (int s = 0; s < pieces; s++) {
        double t0 = (double)s / pieces, t1 = (double)(s + 1) / pieces;
        double ax = sx0 + ex * t0, ay = sy0 + ey * t0, bx = sx0 + ex * t1, by = sy0 + ey * t1;
        double lx = fmin(ax, bx) - 1.0, hx = fmax(ax, bx) + 1.0;
        double ly = fmin(ay, by) - 1.0, hy = fmax(ay, by) + 1.0;
        int cx0 = (int)floor((lx - (double)o->gx0) / (double)o->gcs);
        int cx1 = (int)floor((hx - (double)o->gx0) / (double)o->gcs);
        int cy0 = (int)floor((ly - (double)o->gy0) / (double)o->gcs);
        int cy1 = (int)floor((hy - (double)o->gy0) / (double)o->gcs);
        if (cx0 < 0) cx0 = 0;
        if (cy0 < 0) cy0 = 0;
        if (cx1 >= o->gnx) cx1 = o->gnx - 1;
        if (cy1 >= o->gny) cy1 = o->gny - 1;
        for (int cy = cy0; cy <= cy1; cy++)
            for (int cx = cx0; cx <= cx1; cx++) {
                int c = cy * o->gnx + cx;
                for (int it = o->gstart[c]; it < o->gstart[c + 1]; it++) {
                    int k = o->gitems[it];
                    if (stamp[k] == *tick) continue;
                    stamp[k] = *tick;
                    if (o->bx1[k] < qx_lo || o->bx0[k] > qx_hi || o->by1[k] < qy_lo ||
                        o->by0[k] > qy_hi)
                        continue;
                    if (blocked_by_poly(o, k, px, py, Dx, Dy, U)) return 1;
                }
            }
    }
    return 0;
}

static int vis_points(const orc_t *o, ll ax, ll ay, ll bx, ll by, int *stamp, int *tick) {
    frac_t one = {1, 1};
    if (ax == bx && ay == by) return 1;
    return !segment_blocked(o, ax, ay, bx - ax, by - ay, one, stamp, tick);
}

/* Segment source s, query point q: returns 1 and the exact foot data when the
 * perpendicular foot lies strictly inside the segment (Sec. 4 distance rule)
 * and q sees it. */
static int seg_foot_interior(const orc_t *o, int s, ll qx, ll qy, ll *num, ll *den, ll *side) {
    const ll *L = o->sl + 4 * s;
    ll ux = L[2] - L[0], uy = L[3] - L[1];
    *num = (qx - L[0]) * ux + (qy - L[1]) * uy;
    *den = ux * ux + uy * uy;
    *side = cross2(ux, uy, qx - L[0], qy - L[1]);
    return *num > 0 && *num < *den;
}

static int vis_foot(const orc_t *o, int s, ll qx, ll qy, ll side, ll den, int *stamp, int *tick) {
    /* q - foot = (side/den) * perp(u) with perp(u) = (-uy, ux): the points
     * q + v*D, D = -side*perp(u), v in (0, 1/den) are the open segment q->foot. */
    const ll *L = o->sl + 4 * s;
    ll ux = L[2] - L[0], uy = L[3] - L[1];
    if (side == 0) return 1; /* q on the segment: zero-length leg */
    /* the open segment q -> foot is q + v * D, D = -sgn(side) perp(u), for
     * v in (0, |side| / den): both bounded by the lattice, so the rational
     * comparisons stay within __int128 */
    const ll sg = side > 0 ? 1 : -1;
    ll Dx = sg * uy, Dy = -sg * ux;
    frac_t U = {side > 0 ? side : -side, den};
    return !segment_blocked(o, qx, qy, Dx, Dy, U, stamp, tick);
}

/* ------------------------------------------------------------------------ */
/* cones                                                                    */
/* ------------------------------------------------------------------------ */

/* Shadow cone of vertex generator v arriving along direction (dx, dy): the
 * path turns around the obstacle toward it, so departures lie between the
 * extension of the arrival direction and the first obstacle edge met when
 * rotating toward the obstacle. Empty if the arrival points into the wedge. */
static void set_cone(orc_t *o, int v, ll dx, ll dy) {
    o->cdx[v] = dx;
    o->cdy[v] = dy;
    int a = sgn(cross2(dx, dy, o->wsx[v], o->wsy[v]));
    int b = sgn(cross2(dx, dy, o->wex[v], o->wey[v]));
    if (a >= 0 && b >= 0 && (a | b))
        o->cside[v] = CONE_LEFT;
    else if (a <= 0 && b <= 0 && (a | b))
        o->cside[v] = CONE_RIGHT;
    else
        o->cside[v] = CONE_EMPTY;
}

static int in_cone(const orc_t *o, int v, ll wx, ll wy) {
    ll dx = o->cdx[v], dy = o->cdy[v];
    switch (o->cside[v]) {
    case CONE_NONE:
        return 1;
    case CONE_LEFT: { /* between d and wedge start, rotating counter-clockwise */
        ll ex = o->wsx[v], ey = o->wsy[v];
        if (cross2(dx, dy, ex, ey) == 0) /* edge continues straight on: a ray */
            return cross2(dx, dy, wx, wy) == 0 && dx * wx + dy * wy >= 0;
        return cross2(dx, dy, wx, wy) >= 0 && cross2(wx, wy, ex, ey) >= 0;
    }
    case CONE_RIGHT: { /* between wedge end and d, rotating clockwise */
        ll ex = o->wex[v], ey = o->wey[v];
        if (cross2(dx, dy, ex, ey) == 0)
            return cross2(dx, dy, wx, wy) == 0 && dx * wx + dy * wy >= 0;
        return cross2(dx, dy, wx, wy) <= 0 && cross2(wx, wy, ex, ey) <= 0;
    }
    default:
        return 0;
    }
}

/* ------------------------------------------------------------------------ */
/* scene setup                                                              */
/* ------------------------------------------------------------------------ */

static int fail(orc_t *o, int code, const char *msg) {
    snprintf(o->err, sizeof o->err, "%s", msg);
    return code;
}

/* angle classification relative to reference direction r: 0 for [0, pi), 1 for [pi, 2pi) */
static int half_rel(ll rx, ll ry, ll x, ll y) {
    ll c = cross2(rx, ry, x, y);
    if (c > 0) return 0;
    if (c < 0) return 1;
    return (rx * x + ry * y > 0) ? 0 : 1;
}
/* -1, 0, +1: angle of a relative to r compared with angle of b relative to r */
static int ang_cmp(ll rx, ll ry, ll ax, ll ay, ll bx, ll by) {
    int ha = half_rel(rx, ry, ax, ay), hb = half_rel(rx, ry, bx, by);
    if (ha != hb) return ha < hb ? -1 : 1;
    ll c = cross2(ax, ay, bx, by);
    return c > 0 ? -1 : (c < 0 ? 1 : 0);
}

/* direction x inside the closed sector [s, e] (CCW, angle in (0, pi]) */
static int in_sector(ll sx, ll sy, ll ex, ll ey, ll x, ll y) {
    if (cross2(sx, sy, ex, ey) == 0) /* half-plane: angle pi */
        return cross2(sx, sy, x, y) >= 0;
    return cross2(sx, sy, x, y) >= 0 && cross2(x, y, ex, ey) >= 0;
}

/* Union of closed angular sectors [s_k, e_k] (CCW, each of angle in (0, pi]).
 * Returns 1 with the union in (us, ue) if it is one arc of angle < pi,
 * 0 if it is connected but not such an arc, -1 if it is not connected. */
static int sector_union(int m, const ll *s, const ll *e, ll *us, ll *ue) {
    /* connectivity: sectors touch when one contains the other's start */
    int comp[64];
    for (int k = 0; k < m; k++) comp[k] = k;
    for (int changed = 1; changed;) {
        changed = 0;
        for (int a = 0; a < m; a++)
            for (int b = 0; b < m; b++) {
                if (comp[a] == comp[b]) continue;
                if (in_sector(s[2 * a], s[2 * a + 1], e[2 * a], e[2 * a + 1], s[2 * b], s[2 * b + 1]) ||
                    in_sector(s[2 * b], s[2 * b + 1], e[2 * b], e[2 * b + 1], s[2 * a], s[2 * a + 1])) {
                    int lo = comp[a] < comp[b] ? comp[a] : comp[b];
                    comp[a] = comp[b] = lo;
                    changed = 1;
                }
            }
    }
    for (int k = 0; k < m; k++)
        if (comp[k] != comp[0]) return -1;
    /* a start not covered by any other sector's interior-or-start is the union's start */
    for (int a = 0; a < m; a++) {
        ll rx = s[2 * a], ry = s[2 * a + 1];
        int ok = 1;
        for (int k = 0; k < m && ok; k++)
            if (ang_cmp(rx, ry, s[2 * k], s[2 * k + 1], e[2 * k], e[2 * k + 1]) > 0) ok = 0;
        if (!ok) continue;
        ll ceX = e[2 * a], ceY = e[2 * a + 1];
        for (int k = 0; k < m; k++)
            if (ang_cmp(rx, ry, e[2 * k], e[2 * k + 1], ceX, ceY) > 0) { ceX = e[2 * k]; ceY = e[2 * k + 1]; }
        if (cross2(rx, ry, ceX, ceY) > 0) {
            us[0] = rx; us[1] = ry;
            ue[0] = ceX; ue[1] = ceY;
            return 1;
        }
        return 0;
    }
    return 0; /* connected and wrapping every start: the full circle */
}

static void grid_build(orc_t *o) {
    ll x0 = 0, y0 = 0, x1 = o->Wx * o->S, y1 = o->Wy * o->S;
    for (int k = 0; k < o->np; k++) {
        if (o->bx0[k] < x0) x0 = o->bx0[k];
        if (o->by0[k] < y0) y0 = o->by0[k];
        if (o->bx1[k] > x1) x1 = o->bx1[k];
        if (o->by1[k] > y1) y1 = o->by1[k];
    }
    ll span = (x1 - x0 > y1 - y0) ? x1 - x0 : y1 - y0;
    int target = (int)sqrt((double)o->np) + 1;
    if (target > 256) target = 256;
    ll cs = span / target + 1;
    o->gx0 = x0 - 1;
    o->gy0 = y0 - 1;
    o->gcs = cs;
    o->gnx = (int)((x1 + 1 - o->gx0) / cs) + 1;
    o->gny = (int)((y1 + 1 - o->gy0) / cs) + 1;
    int nc = o->gnx * o->gny;
    o->gstart = calloc(nc + 1, sizeof(int));
    int *fillp = calloc(nc + 1, sizeof(int));
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            for (int c = 0; c < nc; c++) o->gstart[c + 1] += o->gstart[c];
            o->gitems = malloc(sizeof(int) * (o->gstart[nc] + 1));
        }
        for (int k = 0; k < o->np; k++) {
            int cx0 = (int)((o->bx0[k] - o->gx0) / cs), cx1 = (int)((o->bx1[k] - o->gx0) / cs);
            int cy0 = (int)((o->by0[k] - o->gy0) / cs), cy1 = (int)((o->by1[k] - o->gy0) / cs);
            for (int cy = cy0; cy <= cy1; cy++)
                for (int cx = cx0; cx <= cx1; cx++) {
                    int c = cy * o->gnx + cx;
                    if (pass == 0)
                        o->gstart[c + 1]++;
                    else
                        o->gitems[o->gstart[c] + fillp[c]++] = k;
                }
        }
    }
    free(fillp);
}

static int cmp_pos(const void *a, const void *b) {
    const ll *x = a, *y = b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    return x[2] < y[2] ? -1 : (x[2] > y[2]);
}

/* A source coordinate on the lattice, rounded half to even: to the coarser
 * "pixel" lattice Sp (then scaled to S), or to S itself when snapping fine. */
static ll snap_source(const orc_t *o, double x) {
    if (!o->fine && o->Sp) return (ll)nearbyint(x * (double)o->Sp) * (o->S / o->Sp);
    return (ll)nearbyint(x * (double)o->S);
}

/* pixel centre on the lattice: (2i+1) * S * W / (2N) */
static ll pix_lat(ll S, ll W, int N, int i) { return (2 * (ll)i + 1) * S * W / (2 * (ll)N); }

static int build(orc_t *o, ll Wx, ll Wy, int Nx, int Ny, int np, const int *poff,
                 const int *pxy, int npt, const double *pts, int nseg, const double *segs) {
    if (Wx <= 0 || Wy <= 0 || Nx <= 0 || Ny <= 0 || np < 0 || npt < 0 || nseg < 0)
        return fail(o, O_EARG, "bad sizes");
    if (npt + nseg == 0) return fail(o, O_EARG, "no sources");
    o->Wx = Wx; o->Wy = Wy; o->Nx = Nx; o->Ny = Ny;
    /* lattice scale */
    ll S = 1;
    while (((S * Wx) % (2 * (ll)Nx)) || ((S * Wy) % (2 * (ll)Ny))) {
        S *= 2;
        if (S > 32768) return fail(o, O_EGEOM, "pixel centres not on a power-of-two lattice");
    }
    ll mnx = 0, mny = 0, mxx = Wx, mxy = Wy;
    for (int i = 0; i < (np ? poff[np] : 0); i++) {
        ll x = pxy[2 * i], y = pxy[2 * i + 1];
        if (x < mnx) mnx = x;
        if (x > mxx) mxx = x;
        if (y < mny) mny = y;
        if (y > mxy) mxy = y;
    }
    ll span = (mxx - mnx > mxy - mny) ? mxx - mnx : mxy - mny;
    if (S * span > (1LL << 24)) return fail(o, O_EGEOM, "scene too large for the exact lattice");
    ll Sp = 0; /* the coarser lattice of "pixel" snapping */
    if (S * span <= 32767)
        for (Sp = S; 2 * Sp * span <= 32767;) Sp *= 2;
    while (2 * S * span <= (1LL << 24)) S *= 2;
    o->S = S;
    o->Sp = Sp;
    /* polygons */
    o->np = np;
    o->po = malloc(sizeof(int) * (np + 1));
    int nv = np ? poff[np] : 0;
    o->px = malloc(sizeof(ll) * (nv + 1));
    o->py = malloc(sizeof(ll) * (nv + 1));
    o->bx0 = malloc(sizeof(ll) * (np + 1)); o->by0 = malloc(sizeof(ll) * (np + 1));
    o->bx1 = malloc(sizeof(ll) * (np + 1)); o->by1 = malloc(sizeof(ll) * (np + 1));
    o->po[0] = 0;
    for (int k = 0; k < np; k++) {
        int b = poff[k], e = poff[k + 1], m = e - b;
        if (m < 3 || b < 0 || e < b) return fail(o, O_EGEOM, "polygon with < 3 vertices");
        ll area2 = 0;
        for (int i = 0; i < m; i++) {
            int j = (i + 1) % m;
            area2 += (ll)pxy[2 * (b + i)] * pxy[2 * (b + j) + 1] -
                     (ll)pxy[2 * (b + j)] * pxy[2 * (b + i) + 1];
        }
        if (area2 == 0) return fail(o, O_EGEOM, "degenerate polygon");
        for (int i = 0; i < m; i++) {
            int src = area2 > 0 ? b + i : b + (m - 1 - i);
            o->px[b + i] = (ll)pxy[2 * src] * S;
            o->py[b + i] = (ll)pxy[2 * src + 1] * S;
        }
        o->po[k + 1] = e;
        ll x0 = o->px[b], x1 = x0, y0 = o->py[b], y1 = y0;
        for (int i = 0; i < m; i++) {
            ll ax = o->px[b + i], ay = o->py[b + i];
            ll bx = o->px[b + (i + 1) % m], by = o->py[b + (i + 1) % m];
            ll cx = o->px[b + (i + 2) % m], cy = o->py[b + (i + 2) % m];
            if (orient(ax, ay, bx, by, cx, cy) <= 0)
                return fail(o, O_EGEOM, "polygon not strictly convex");
            if (ax < x0) x0 = ax;
            if (ax > x1) x1 = ax;
            if (ay < y0) y0 = ay;
            if (ay > y1) y1 = ay;
        }
        o->bx0[k] = x0; o->bx1[k] = x1; o->by0[k] = y0; o->by1[k] = y1;
    }
    grid_build(o);
    /* generators */
    int cap = npt + 3 * nseg + nv;
    o->kind = malloc(sizeof(int) * cap); o->sidx = malloc(sizeof(int) * cap);
    o->tx = malloc(sizeof(double) * cap); o->ty = malloc(sizeof(double) * cap);
    o->lx = malloc(sizeof(ll) * cap); o->ly = malloc(sizeof(ll) * cap);
    o->wsx = calloc(cap, sizeof(ll)); o->wsy = calloc(cap, sizeof(ll));
    o->wex = calloc(cap, sizeof(ll)); o->wey = calloc(cap, sizeof(ll));
    o->cost = malloc(sizeof(double) * cap); o->par = malloc(sizeof(int) * cap);
    o->cdx = calloc(cap, sizeof(ll)); o->cdy = calloc(cap, sizeof(ll));
    o->cside = calloc(cap, sizeof(int));
    int g = 0;
    int *stamp = calloc(np + 1, sizeof(int));
    int tick = 0;
#define FREE_CHECK(LX, LY, MSG)                                                          \
    do {                                                                                 \
        if ((LX) < 0 || (LY) < 0 || (LX) > Wx * S || (LY) > Wy * S)                      \
            return fail(o, O_EGEOM, MSG " outside the world");                            \
        for (int kk = 0; kk < np; kk++) {                                                \
            int bb = o->po[kk], mm = o->po[kk + 1] - bb, inside = 1;                       \
            for (int ii = 0; ii < mm && inside; ii++)                                    \
                if (orient(o->px[bb + ii], o->py[bb + ii], o->px[bb + (ii + 1) % mm],      \
                           o->py[bb + (ii + 1) % mm], (LX), (LY)) < 0)                    \
                    inside = 0;                                                          \
            if (inside) return fail(o, O_EGEOM, MSG " not strictly free");               \
        }                                                                                \
    } while (0)
    for (int i = 0; i < npt; i++) {
        o->kind[g] = K_POINT; o->sidx[g] = i;
        o->tx[g] = pts[2 * i]; o->ty[g] = pts[2 * i + 1];
        o->lx[g] = snap_source(o, pts[2 * i]);
        o->ly[g] = snap_source(o, pts[2 * i + 1]);
        FREE_CHECK(o->lx[g], o->ly[g], "point source");
        g++;
    }
    o->nseg = nseg;
    o->sf = malloc(sizeof(double) * 4 * (nseg + 1));
    o->sl = malloc(sizeof(ll) * 4 * (nseg + 1));
    for (int s = 0; s < nseg; s++) {
        for (int c = 0; c < 4; c++) {
            o->sf[4 * s + c] = segs[4 * s + c];
            o->sl[4 * s + c] = snap_source(o, segs[4 * s + c]);
        }
        if (o->sl[4 * s] == o->sl[4 * s + 2] && o->sl[4 * s + 1] == o->sl[4 * s + 3])
            return fail(o, O_EGEOM, "zero-length segment source");
        FREE_CHECK(o->sl[4 * s], o->sl[4 * s + 1], "segment endpoint");
        FREE_CHECK(o->sl[4 * s + 2], o->sl[4 * s + 3], "segment endpoint");
        /* the whole closed segment must avoid every closed obstacle */
        for (int k = 0; k < np; k++) {
            int b = o->po[k], m = o->po[k + 1] - b, sep = 0;
            ll ax = o->sl[4 * s], ay = o->sl[4 * s + 1], bx = o->sl[4 * s + 2], by = o->sl[4 * s + 3];
            for (int i = 0; i < m && !sep; i++) { /* polygon edge line separates? */
                ll ex = o->px[b + i], ey = o->py[b + i];
                ll fx = o->px[b + (i + 1) % m], fy = o->py[b + (i + 1) % m];
                if (orient(ex, ey, fx, fy, ax, ay) < 0 && orient(ex, ey, fx, fy, bx, by) < 0) sep = 1;
            }
            if (!sep) { /* segment line separates? */
                int pos = 0, neg = 0;
                for (int i = 0; i < m; i++) {
                    ll v = orient(ax, ay, bx, by, o->px[b + i], o->py[b + i]);
                    pos |= v > 0; neg |= v < 0;
                    if (v == 0) { pos = neg = 1; }
                }
                sep = !(pos && neg);
            }
            if (!sep) return fail(o, O_EGEOM, "segment source touches an obstacle");
        }
        for (int c = 0; c < 3; c++) {
            o->kind[g] = K_SEGA + c; o->sidx[g] = s;
            int off = (c == 1) ? 2 : 0;
            o->tx[g] = segs[4 * s + off]; o->ty[g] = segs[4 * s + off + 1];
            o->lx[g] = o->sl[4 * s + off]; o->ly[g] = o->sl[4 * s + off + 1];
            g++;
        }
    }
    o->nsrc = g;
    o->vbase = g;
    /* obstacle vertices: convex corners of the union of closed obstacles,
       polygon-major input order, first occurrence of a position kept */
    ll *keys = malloc(sizeof(ll) * 3 * (nv + 1));
    for (int i = 0; i < nv; i++) { keys[3 * i] = o->px[i]; keys[3 * i + 1] = o->py[i]; keys[3 * i + 2] = i; }
    qsort(keys, nv, 3 * sizeof(ll), cmp_pos);
    char *first = calloc(nv + 1, 1);
    for (int i = 0; i < nv; i++)
        if (i == 0 || keys[3 * i] != keys[3 * (i - 1)] || keys[3 * i + 1] != keys[3 * (i - 1) + 1])
            first[keys[3 * i + 2]] = 1;
    free(keys);
    for (int k = 0; k < np; k++) {
        int b = o->po[k], m = o->po[k + 1] - b;
        for (int i = 0; i < m; i++) {
            int vi = b + i;
            if (!first[vi]) continue;
            ll vx = o->px[vi], vy = o->py[vi];
            ll ss[128], ee[128];
            int ns = 0, inside = 0;
            int cx = (int)((vx - o->gx0) / o->gcs), cy = (int)((vy - o->gy0) / o->gcs);
            tick++;
            for (int dyc = -1; dyc <= 1 && !inside; dyc++)
                for (int dxc = -1; dxc <= 1 && !inside; dxc++) {
                    int ccx = cx + dxc, ccy = cy + dyc;
                    if (ccx < 0 || ccy < 0 || ccx >= o->gnx || ccy >= o->gny) continue;
                    int c = ccy * o->gnx + ccx;
                    for (int it = o->gstart[c]; it < o->gstart[c + 1] && !inside; it++) {
                        int q = o->gitems[it];
                        if (stamp[q] == tick) continue;
                        stamp[q] = tick;
                        if (vx < o->bx0[q] || vx > o->bx1[q] || vy < o->by0[q] || vy > o->by1[q]) continue;
                        int qb = o->po[q], qm = o->po[q + 1] - qb, zeros = 0, neg = 0, zi = -1;
                        for (int j = 0; j < qm; j++) {
                            ll v = orient(o->px[qb + j], o->py[qb + j], o->px[qb + (j + 1) % qm],
                                          o->py[qb + (j + 1) % qm], vx, vy);
                            if (v < 0) neg = 1;
                            if (v == 0) { zeros++; zi = j; }
                        }
                        if (neg) continue;
                        if (zeros == 0) { inside = 1; break; }
                        int vert = -1;
                        for (int j = 0; j < qm; j++)
                            if (o->px[qb + j] == vx && o->py[qb + j] == vy) vert = j;
                        if (ns >= 64) return fail(o, O_EGEOM, "too many obstacles meet at a vertex");
                        if (vert >= 0) {
                            int nx = qb + (vert + 1) % qm, pv = qb + (vert + qm - 1) % qm;
                            ss[2 * ns] = o->px[nx] - vx; ss[2 * ns + 1] = o->py[nx] - vy;
                            ee[2 * ns] = o->px[pv] - vx; ee[2 * ns + 1] = o->py[pv] - vy;
                        } else {
                            ll ex = o->px[qb + (zi + 1) % qm] - o->px[qb + zi];
                            ll ey = o->py[qb + (zi + 1) % qm] - o->py[qb + zi];
                            ss[2 * ns] = ex; ss[2 * ns + 1] = ey;
                            ee[2 * ns] = -ex; ee[2 * ns + 1] = -ey;
                        }
                        ns++;
                    }
                }
            if (inside) continue;
            ll us[2], ue[2];
            int r = sector_union(ns, ss, ee, us, ue);
            if (r < 0) return fail(o, O_EGEOM, "obstacles touch at a single point");
            if (r == 0) continue;
            o->kind[g] = K_VERT; o->sidx[g] = vi;
            o->lx[g] = vx; o->ly[g] = vy;
            o->tx[g] = (double)(vx / S); o->ty[g] = (double)(vy / S);
            o->wsx[g] = us[0]; o->wsy[g] = us[1]; o->wex[g] = ue[0]; o->wey[g] = ue[1];
            g++;
        }
    }
    free(first);
    free(stamp);
    o->ng = g;
    o->nvert = g - o->vbase;
    return O_OK;
#undef FREE_CHECK
}

/* ------------------------------------------------------------------------ */
/* vertex costs (Dijkstra over the visibility graph)                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    orc_t *o;
    int next;  /* shared row counter, taken with an atomic add */
    int chunk;
} vis_job;

static int gen_sees_vertex(const orc_t *o, int u, int v, int *stamp, int *tick) {
    if (o->kind[u] == K_SEGI) {
        ll num, den, side;
        if (!seg_foot_interior(o, o->sidx[u], o->lx[v], o->ly[v], &num, &den, &side)) return 0;
        return vis_foot(o, o->sidx[u], o->lx[v], o->ly[v], side, den, stamp, tick);
    }
    return vis_points(o, o->lx[u], o->ly[u], o->lx[v], o->ly[v], stamp, tick);
}

static void *vis_worker(void *arg) {
    vis_job *j = arg;
    orc_t *o = j->o;
    int *stamp = calloc(o->np + 1, sizeof(int));
    int tick = 0;
    for (;;) {
        int u0 = __atomic_fetch_add(&j->next, j->chunk, __ATOMIC_RELAXED);
        if (u0 >= o->ng) break;
        int u1 = u0 + j->chunk > o->ng ? o->ng : u0 + j->chunk;
        for (int u = u0; u < u1; u++)
            for (int vv = 0; vv < o->nvert; vv++) {
                int v = o->vbase + vv;
                if (v == u) continue;
                if (o->kind[u] == K_VERT && v < u) continue; /* symmetric: upper triangle */
                int s = gen_sees_vertex(o, u, v, stamp, &tick);
                o->vis[(size_t)u * o->nvert + vv] = (unsigned char)s;
                if (o->kind[u] == K_VERT) o->vis[(size_t)v * o->nvert + (u - o->vbase)] = (unsigned char)s;
            }
    }
    free(stamp);
    return NULL;
}

static double gen_len(const orc_t *o, int u, int v) {
    if (o->kind[u] == K_SEGI) {
        const double *F = o->sf + 4 * o->sidx[u];
        double ux = F[2] - F[0], uy = F[3] - F[1];
        double c = ux * (o->ty[v] - F[1]) - uy * (o->tx[v] - F[0]);
        return fabs(c) / sqrt(ux * ux + uy * uy);
    }
    double dx = o->tx[v] - o->tx[u], dy = o->ty[v] - o->ty[u];
    return sqrt(dx * dx + dy * dy);
}

/* arrival direction at v when its parent is u */
static void arrival_dir(const orc_t *o, int u, int v, ll *dx, ll *dy) {
    if (o->kind[u] == K_SEGI) {
        const ll *L = o->sl + 4 * o->sidx[u];
        ll ux = L[2] - L[0], uy = L[3] - L[1];
        ll side = cross2(ux, uy, o->lx[v] - L[0], o->ly[v] - L[1]);
        *dx = (side > 0) ? -uy : uy; /* perp(u) = (-uy, ux) signed toward v */
        *dy = (side > 0) ? ux : -ux;
        return;
    }
    *dx = o->lx[v] - o->lx[u];
    *dy = o->ly[v] - o->ly[u];
}

typedef struct { double c; int id; } hitem;
static int h_less(hitem a, hitem b) { return a.c < b.c || (a.c == b.c && a.id < b.id); }
static void h_push(hitem *h, int *n, hitem x) {
    int i = (*n)++;  /* caller guarantees capacity */
    h[i] = x;
    while (i > 0) {
        int p = (i - 1) / 2;
        if (!h_less(h[i], h[p])) break;
        hitem t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}
static hitem h_pop(hitem *h, int *n) {
    hitem r = h[0];
    h[0] = h[--(*n)];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, rr = l + 1, m = i;
        if (l < *n && h_less(h[l], h[m])) m = l;
        if (rr < *n && h_less(h[rr], h[m])) m = rr;
        if (m == i) break;
        hitem t = h[i]; h[i] = h[m]; h[m] = t;
        i = m;
    }
    return r;
}

static int vertex_costs(orc_t *o, int nthreads, int use_cone) {
    size_t nvis = (size_t)o->ng * (o->nvert ? o->nvert : 1);
    o->vis = calloc(nvis, 1);
    if (!o->vis) return fail(o, O_ENOMEM, "visibility matrix");
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    vis_job job = {o, 0, 8};
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, vis_worker, &job);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    for (int g = 0; g < o->ng; g++) {
        o->cost[g] = INFINITY;
        o->par[g] = -1;
        o->cside[g] = (g < o->nsrc) ? CONE_NONE : CONE_EMPTY;
    }
    char *done = calloc(o->ng, 1);
    size_t hcap = (size_t)o->ng * 4 + 64;
    hitem *heap = malloc(sizeof(hitem) * hcap);
    int hn = 0;
    for (int g = 0; g < o->nsrc; g++) {
        o->cost[g] = 0.0;
        o->par[g] = g;
        h_push(heap, &hn, (hitem){0.0, g});
    }
    while (hn > 0) {
        hitem it = h_pop(heap, &hn);
        int u = it.id;
        if (done[u] || it.c != o->cost[u]) continue;
        done[u] = 1;
        if (o->kind[u] == K_VERT) {
            ll dx, dy;
            arrival_dir(o, o->par[u], u, &dx, &dy);
            set_cone(o, u, dx, dy);
        }
        for (int vv = 0; vv < o->nvert; vv++) {
            int v = o->vbase + vv;
            if (done[v] || !o->vis[(size_t)u * o->nvert + vv]) continue;
            if (use_cone && o->kind[u] == K_VERT &&
                !in_cone(o, u, o->lx[v] - o->lx[u], o->ly[v] - o->ly[u]))
                continue;
            double c = o->cost[u] + gen_len(o, u, v);
            if (c < o->cost[v] || (c == o->cost[v] && u < o->par[v])) {
                o->cost[v] = c;
                o->par[v] = u;
                if ((size_t)hn + 1 >= hcap) {
                    hcap *= 2;
                    heap = realloc(heap, sizeof(hitem) * hcap);
                }
                h_push(heap, &hn, (hitem){c, v});
            }
        }
    }
    if (!use_cone)
        for (int g = o->vbase; g < o->ng; g++)
            if (o->par[g] >= 0) {
                ll dx, dy;
                arrival_dir(o, o->par[g], g, &dx, &dy);
                set_cone(o, g, dx, dy);
            }
    free(done);
    free(heap);
    return O_OK;
}

/* ------------------------------------------------------------------------ */
/* pixel field                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    const orc_t *o;
    int n, next, blk;  /* pixels, shared block counter, block size */
    const int *ij;
    double *dist, *second;
    int *par, *par2;
    int use_cone;
} pix_job;

static int pixel_free(const orc_t *o, ll px, ll py) {
    int cx = (int)((px - o->gx0) / o->gcs), cy = (int)((py - o->gy0) / o->gcs);
    if (cx < 0 || cy < 0 || cx >= o->gnx || cy >= o->gny) return 1;
    int c = cy * o->gnx + cx;
    for (int it = o->gstart[c]; it < o->gstart[c + 1]; it++) {
        int k = o->gitems[it];
        int b = o->po[k], m = o->po[k + 1] - b, inside = 1;
        for (int i = 0; i < m && inside; i++)
            if (orient(o->px[b + i], o->py[b + i], o->px[b + (i + 1) % m], o->py[b + (i + 1) % m], px, py) <= 0)
                inside = 0;
        if (inside) return 0;
    }
    return 1;
}

/* The field at one point: lattice position (px, py) for the exact predicates,
 * world coordinates (fx, fy) for the distances. Best and second-best valid
 * generator (different ids), by key then id. */
static void eval_point(const orc_t *o, ll px, ll py, double fx, double fy, hitem *heap, int *stamp, int *tick,
                       int use_cone, double *d1, int *p1, double *d2, int *p2) {
    *d1 = *d2 = INFINITY;
    *p1 = *p2 = -1;
    if (!pixel_free(o, px, py)) return;
    int hn = 0;
    for (int g = 0; g < o->ng; g++) {
        if (!(o->cost[g] < INFINITY)) continue;
        double key;
        if (o->kind[g] == K_SEGI) {
            ll num, den, side;
            if (!seg_foot_interior(o, o->sidx[g], px, py, &num, &den, &side)) continue;
            const double *F = o->sf + 4 * o->sidx[g];
            double ux = F[2] - F[0], uy = F[3] - F[1];
            key = fabs(ux * (fy - F[1]) - uy * (fx - F[0])) / sqrt(ux * ux + uy * uy);
        } else {
            if (o->kind[g] == K_VERT && use_cone && !in_cone(o, g, px - o->lx[g], py - o->ly[g]))
                continue;
            double dx = fx - o->tx[g], dy = fy - o->ty[g];
            key = o->cost[g] + sqrt(dx * dx + dy * dy);
        }
        heap[hn++] = (hitem){key, g};
    }
    for (int k = hn / 2 - 1; k >= 0; k--) { /* heapify */
        int i2 = k;
        for (;;) {
            int l = 2 * i2 + 1, r = l + 1, m = i2;
            if (l < hn && h_less(heap[l], heap[m])) m = l;
            if (r < hn && h_less(heap[r], heap[m])) m = r;
            if (m == i2) break;
            hitem t = heap[i2]; heap[i2] = heap[m]; heap[m] = t;
            i2 = m;
        }
    }
    int found = 0;
    while (hn > 0 && found < 2) {
        hitem it = h_pop(heap, &hn);
        int g = it.id, ok;
        if (o->kind[g] == K_SEGI) {
            ll num, den, side;
            seg_foot_interior(o, o->sidx[g], px, py, &num, &den, &side);
            ok = vis_foot(o, o->sidx[g], px, py, side, den, stamp, tick);
        } else {
            ok = vis_points(o, px, py, o->lx[g], o->ly[g], stamp, tick);
        }
        if (!ok) continue;
        if (found == 0) { *d1 = it.c; *p1 = g; }
        else { *d2 = it.c; *p2 = g; }
        found++;
    }
}

static void eval_pixel(const orc_t *o, int i, int j, hitem *heap, int *stamp, int *tick,
                       int use_cone, double *d1, int *p1, double *d2, int *p2) {
    ll px = pix_lat(o->S, o->Wx, o->Nx, i), py = pix_lat(o->S, o->Wy, o->Ny, j);
    double fx = ((double)i + 0.5) * (double)o->Wx / (double)o->Nx;
    double fy = ((double)j + 0.5) * (double)o->Wy / (double)o->Ny;
    eval_point(o, px, py, fx, fy, heap, stamp, tick, use_cone, d1, p1, d2, p2);
}

static void *pix_worker(void *arg) {
    pix_job *j = arg;
    const orc_t *o = j->o;
    hitem *heap = malloc(sizeof(hitem) * (o->ng + 1));
    int *stamp = calloc(o->np + 1, sizeof(int));
    int tick = 0;
    for (;;) {
        int n0 = __atomic_fetch_add(&j->next, j->blk, __ATOMIC_RELAXED);
        if (n0 >= j->n) break;
        int n1 = n0 + j->blk > j->n ? j->n : n0 + j->blk;
        for (int n = n0; n < n1; n++) {
            double d2;
            int p2;
            eval_pixel(o, j->ij[2 * n], j->ij[2 * n + 1], heap, stamp, &tick, j->use_cone,
                       &j->dist[n], &j->par[n], &d2, &p2);
            if (j->second) j->second[n] = d2;
            if (j->par2) j->par2[n] = p2;
        }
    }
    free(heap);
    free(stamp);
    return NULL;
}

/* ------------------------------------------------------------------------ */
/* exported API (ctypes)                                                    */
/* ------------------------------------------------------------------------ */

static void orc_free_inner(orc_t *o) {
    void *ps[] = {o->po, o->px, o->py, o->bx0, o->by0, o->bx1, o->by1, o->sf, o->sl,
                  o->kind, o->sidx, o->tx, o->ty, o->lx, o->ly, o->wsx, o->wsy, o->wex,
                  o->wey, o->cost, o->par, o->cdx, o->cdy, o->cside, o->gstart, o->gitems,
                  o->vis};
    for (size_t i = 0; i < sizeof ps / sizeof ps[0]; i++) free(ps[i]);
}

void orc_free(void *h) {
    if (!h) return;
    orc_free_inner((orc_t *)h);
    free(h);
}

/* Builds the scene and the vertex costs. use_cone = 0 relaxes every visible
 * edge (textbook Dijkstra), 1 restricts vertex generators to their cones.
 * snap_fine = 1 rounds sources to the full lattice, 0 to the coarser one. */
void *orc_create(long long Wx, long long Wy, int Nx, int Ny, int np, const int *poff,
                 const int *pxy, int npt, const double *pts, int nseg, const double *segs,
                 int nthreads, int use_cone, int snap_fine, int *status, char *errbuf, int errlen) {
    orc_t *o = calloc(1, sizeof(orc_t));
    o->fine = snap_fine != 0;
    int st = build(o, Wx, Wy, Nx, Ny, np, poff, pxy, npt, pts, nseg, segs);
    if (st == O_OK) st = vertex_costs(o, nthreads, use_cone);
    if (status) *status = st;
    if (st != O_OK) {
        if (errbuf && errlen > 0) snprintf(errbuf, errlen, "%s", o->err);
        orc_free(o);
        return NULL;
    }
    return o;
}

void orc_info(void *h, int *out) {
    orc_t *o = h;
    out[0] = o->ng; out[1] = o->nsrc; out[2] = o->nvert; out[3] = (int)o->S;
    out[4] = o->np; out[5] = (int)o->Sp;
}

/* generator table: kind, source index (segment / vertex index), lattice xy,
 * true xy, cost, parent, cone side, cone direction, wedge */
void orc_generators(void *h, int *kind, int *sidx, long long *lxy, double *txy, double *cost,
                    int *par, int *cside, long long *cdir, long long *wedge) {
    orc_t *o = h;
    for (int g = 0; g < o->ng; g++) {
        if (kind) kind[g] = o->kind[g];
        if (sidx) sidx[g] = o->sidx[g];
        if (lxy) { lxy[2 * g] = o->lx[g]; lxy[2 * g + 1] = o->ly[g]; }
        if (txy) { txy[2 * g] = o->tx[g]; txy[2 * g + 1] = o->ty[g]; }
        if (cost) cost[g] = o->cost[g];
        if (par) par[g] = o->par[g];
        if (cside) cside[g] = o->cside[g];
        if (cdir) { cdir[2 * g] = o->cdx[g]; cdir[2 * g + 1] = o->cdy[g]; }
        if (wedge) {
            wedge[4 * g] = o->wsx[g]; wedge[4 * g + 1] = o->wsy[g];
            wedge[4 * g + 2] = o->wex[g]; wedge[4 * g + 3] = o->wey[g];
        }
    }
}

/* Field at n pixels (ij = interleaved column, row). dist / parent are the
 * best valid generator, second / par2 the best valid generator with a
 * different id (near-tie detection). use_cone as in orc_create. */
void orc_pixels(void *h, int n, const int *ij, double *dist, int *par, double *second,
                int *par2, int nthreads, int use_cone) {
    orc_t *o = h;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    pix_job job = {o, n, 0, 16, ij, dist, second, par, par2, use_cone};
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, pix_worker, &job);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
}

/* Exact visibility between two lattice points (1 = visible). */
/* Keys of given generators at given pixels: key[n] = cost(g) + |p - g| (the
 * perpendicular distance for a segment interior) when generator g = gen[n] is
 * valid at pixel (i, j) = ij[2n..2n+1] -- the pixel is free, g is reached,
 * p lies in g's shadow cone (obstacle vertices) or its foot strictly inside
 * the segment (segment interiors), and p sees g (or the foot) -- else +inf.
 * The same steps as the per-pixel minimum, for one generator at a time:
 * used to check that a different but tied choice of parent is valid. */
void orc_keys(void *h, int n, const int *ij, const int *gen, double *key) {
    const orc_t *o = h;
    int *stamp = calloc(o->np + 1, sizeof(int));
    int tick = 0;
    for (int q = 0; q < n; q++) {
        const int i = ij[2 * q], j = ij[2 * q + 1], g = gen[q];
        key[q] = INFINITY;
        if (g < 0 || g >= o->ng || !(o->cost[g] < INFINITY)) continue;
        ll px = pix_lat(o->S, o->Wx, o->Nx, i), py = pix_lat(o->S, o->Wy, o->Ny, j);
        if (!pixel_free(o, px, py)) continue;
        double fx = ((double)i + 0.5) * (double)o->Wx / (double)o->Nx;
        double fy = ((double)j + 0.5) * (double)o->Wy / (double)o->Ny;
        double k;
        int ok;
        if (o->kind[g] == K_SEGI) {
            ll num, den, side;
            if (!seg_foot_interior(o, o->sidx[g], px, py, &num, &den, &side)) continue;
            const double *F = o->sf + 4 * o->sidx[g];
            double ux = F[2] - F[0], uy = F[3] - F[1];
            k = fabs(ux * (fy - F[1]) - uy * (fx - F[0])) / sqrt(ux * ux + uy * uy);
            ok = vis_foot(o, o->sidx[g], px, py, side, den, stamp, &tick);
        } else {
            if (o->kind[g] == K_VERT && !in_cone(o, g, px - o->lx[g], py - o->ly[g])) continue;
            double dx = fx - o->tx[g], dy = fy - o->ty[g];
            k = o->cost[g] + sqrt(dx * dx + dy * dy);
            ok = vis_points(o, px, py, o->lx[g], o->ly[g], stamp, &tick);
        }
        if (ok) key[q] = k;
    }
    free(stamp);
}

/* The field at arbitrary lattice points lxy (2 per point), world coordinates
 * lxy / S: best key and generator (the point queries of Sec. 6). */
void orc_points(void *h, int n, const long long *lxy, double *dist, int *par) {
    const orc_t *o = h;
    hitem *heap = malloc(sizeof(hitem) * (o->ng + 1));
    int *stamp = calloc(o->np + 1, sizeof(int));
    int tick = 0;
    for (int q = 0; q < n; q++) {
        double d2;
        int p2;
        eval_point(o, lxy[2 * q], lxy[2 * q + 1], (double)lxy[2 * q] / (double)o->S, (double)lxy[2 * q + 1] / (double)o->S,
                   heap, stamp, &tick, 1, &dist[q], &par[q], &d2, &p2);
    }
    free(heap);
    free(stamp);
}

int orc_visible(void *h, long long ax, long long ay, long long bx, long long by) {
    orc_t *o = h;
    int *stamp = calloc(o->np + 1, sizeof(int));
    int tick = 0;
    int r = vis_points(o, ax, ay, bx, by, stamp, &tick);
    free(stamp);
    return r;
}

int orc_lattice_scale(void *h) { return (int)((orc_t *)h)->S; }

/* Root link of the shortest-path chain at a free, reached pixel: walks the
 * parent chain to its source and returns the root generator, the last point
 * x before it (lattice and true coordinates) and, for a segment interior,
 * the foot parameter t. Returns -1 for unreached pixels. */
int orc_root_link(void *h, int i, int j, int first_parent, double *x_true, double *t_foot) {
    orc_t *o = h;
    if (first_parent < 0) return -1;
    double fx = ((double)i + 0.5) * (double)o->Wx / (double)o->Nx;
    double fy = ((double)j + 0.5) * (double)o->Wy / (double)o->Ny;
    int g = first_parent, guard = 0;
    double xx = fx, xy = fy;
    while (o->kind[g] == K_VERT) {
        xx = o->tx[g];
        xy = o->ty[g];
        g = o->par[g];
        if (g < 0 || ++guard > o->ng + 1) return -1;
    }
    x_true[0] = xx;
    x_true[1] = xy;
    *t_foot = 0.0;
    if (o->kind[g] == K_SEGI) {
        const double *F = o->sf + 4 * o->sidx[g];
        double ux = F[2] - F[0], uy = F[3] - F[1];
        *t_foot = ((xx - F[0]) * ux + (xy - F[1]) * uy) / (ux * ux + uy * uy);
    }
    return g;
}
