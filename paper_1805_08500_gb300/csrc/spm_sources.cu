// spm_sources.cu -- sources moved on the device (dynamic maps, Sec. 6).
//
// A moving source only changes the Source entries of the generator table
// (Sec. 3.1): its lattice point, its true position and, for a segment, its
// lattice and true endpoints. k_update_sources snaps the new coordinates to
// the lattice exactly as scene creation does (round half to even of x * S,
// exact in double for S a power of two), validates them with the same exact
// integer predicates (inside the world, outside every closed obstacle, a
// segment of non-zero length disjoint from every closed obstacle), and
// commits all of them or none: one invalid source leaves the table as it was
// and latches kStBadSource. Being stream-ordered and allocation-free, a frame
// loop of (move sources, compute) runs without host round trips and can be
// captured in a CUDA graph.
#include <cuda_runtime.h>

#include <cstdint>

#include "spm_internal.h"

namespace spm {
namespace {

constexpr int kUpdThreads = 1024;

__device__ __forceinline__ long long orient64(long long ax, long long ay, long long bx, long long by, long long cx,
                                              long long cy) {
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

// One coordinate onto the lattice; false when it is not finite or so large
// that it cannot be inside any world.
__device__ __forceinline__ bool snap(float v, int S, int &out) {
    if (!isfinite(v)) return false;
    const double x = rint((double)v * (double)S);
    if (fabs(x) > 1073741824.0) return false;
    out = (int)x;
    return true;
}

__device__ __forceinline__ bool in_world(const DevScene &ds, int x, int y) {
    return x >= 0 && y >= 0 && (long long)x <= (long long)ds.Wx * ds.S && (long long)y <= (long long)ds.Wy * ds.S;
}

__device__ __forceinline__ int bin_x(const DevScene &ds, int x) {
    const int c = (x - ds.bin_x0) / ds.bin_size;
    return max(0, min(ds.bin_nx - 1, c));
}
__device__ __forceinline__ int bin_y(const DevScene &ds, int y) {
    const int c = (y - ds.bin_y0) / ds.bin_size;
    return max(0, min(ds.bin_ny - 1, c));
}

// Closed convex CCW polygon contains (x, y)?
__device__ __forceinline__ bool closed_contains(const int2 *V, int m, int x, int y) {
    for (int i = 0; i < m; ++i) {
        const int2 a = V[i], b = V[i + 1 == m ? 0 : i + 1];
        if (orient64(a.x, a.y, b.x, b.y, x, y) < 0) return false;
    }
    return true;
}

// Closed segment a-b and closed convex polygon disjoint? Strict separating
// axis: an edge line with both endpoints strictly outside, or the segment's
// line with every vertex strictly on one side.
__device__ __forceinline__ bool seg_clear(const int2 *V, int m, int ax, int ay, int bx, int by) {
    for (int i = 0; i < m; ++i) {
        const int2 p = V[i], q = V[i + 1 == m ? 0 : i + 1];
        if (orient64(p.x, p.y, q.x, q.y, ax, ay) < 0 && orient64(p.x, p.y, q.x, q.y, bx, by) < 0) return true;
    }
    bool pos = false, neg = false, zero = false;
    for (int i = 0; i < m; ++i) {
        const long long o = orient64(ax, ay, bx, by, V[i].x, V[i].y);
        pos |= o > 0;
        neg |= o < 0;
        zero |= o == 0;
    }
    return !zero && !(pos && neg);
}

// Warp-wide: is the world point (x, y) inside or on an obstacle? The lanes
// walk the polygons of its bin.
__device__ bool point_blocked(const DevScene &ds, int x, int y, int lane) {
    const int c = bin_y(ds, y) * ds.bin_nx + bin_x(ds, x);
    bool bad = false;
    for (int it = ds.bin_start[c] + lane; it < ds.bin_start[c + 1]; it += 32) {
        const BinRec r = ds.bin_recs[it];
        if (x < r.box.x || x > r.box.z || y < r.box.y || y > r.box.w) continue;
        bad |= closed_contains(ds.poly_v + r.voff, r.m, x, y);
    }
    return __any_sync(0xffffffffu, bad);
}

// Warp-wide: does the closed segment (both endpoints in the world) touch an
// obstacle? The warp walks the bins under its bounding box, the lanes the
// polygons of each bin.
__device__ bool segment_blocked(const DevScene &ds, int ax, int ay, int bx, int by, int lane) {
    const int x0 = min(ax, bx), x1 = max(ax, bx), y0 = min(ay, by), y1 = max(ay, by);
    const int cx0 = bin_x(ds, x0), cx1 = bin_x(ds, x1), cy0 = bin_y(ds, y0), cy1 = bin_y(ds, y1);
    bool bad = false;
    for (int cy = cy0; cy <= cy1; ++cy)
        for (int cx = cx0; cx <= cx1; ++cx) {
            const int c = cy * ds.bin_nx + cx;
            for (int it = ds.bin_start[c] + lane; it < ds.bin_start[c + 1]; it += 32) {
                const BinRec r = ds.bin_recs[it];
                if (x1 < r.box.x || x0 > r.box.z || y1 < r.box.y || y0 > r.box.w) continue;
                bad |= !seg_clear(ds.poly_v + r.voff, r.m, ax, ay, bx, by);
            }
        }
    return __any_sync(0xffffffffu, bad);
}

// One CTA: every warp validates sources q = warp, warp + 32, ... (all lanes
// of a warp take the same branches: they read the same source), then, if
// every source is valid, the threads write the table.
__global__ void __launch_bounds__(kUpdThreads) k_update_sources(DevScene ds, const float *pts, const float *segs) {
    __shared__ int bad;
    const int np = ds.n_src - 3 * ds.n_seg, ns = ds.n_seg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int q = warp; q < np + ns; q += kUpdThreads / 32) {
        bool ok;
        if (q < np) {
            int x = 0, y = 0;
            ok = snap(pts[2 * q], ds.S, x) && snap(pts[2 * q + 1], ds.S, y) && in_world(ds, x, y);
            if (ok) ok = !point_blocked(ds, x, y, lane);
        } else {
            const int s = q - np;
            int L[4] = {0, 0, 0, 0};
            ok = true;
            for (int c = 0; c < 4; ++c) ok = ok && snap(segs[4 * s + c], ds.S, L[c]);
            ok = ok && !(L[0] == L[2] && L[1] == L[3]) && in_world(ds, L[0], L[1]) && in_world(ds, L[2], L[3]);
            if (ok) ok = !point_blocked(ds, L[0], L[1], lane);
            if (ok) ok = !point_blocked(ds, L[2], L[3], lane);
            if (ok) ok = !segment_blocked(ds, L[0], L[1], L[2], L[3], lane);
        }
        if (!ok && lane == 0) atomicOr(&bad, 1);
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) atomicOr(ds.status, (uint32_t)kStBadSource);
        return;
    }
    int2 *gen_lat = const_cast<int2 *>(ds.gen_lat);
    float2 *gen_pos = const_cast<float2 *>(ds.gen_pos);
    for (int i = threadIdx.x; i < np; i += kUpdThreads) {
        const float fx = pts[2 * i], fy = pts[2 * i + 1];
        int x, y;
        snap(fx, ds.S, x);
        snap(fy, ds.S, y);
        gen_lat[i] = make_int2(x, y);
        gen_pos[i] = make_float2(fx, fy);
    }
    int4 *seg_lat = const_cast<int4 *>(ds.seg_lat);
    float4 *seg_pos = const_cast<float4 *>(ds.seg_pos);
    for (int s = threadIdx.x; s < ns; s += kUpdThreads) {
        const float4 F = make_float4(segs[4 * s], segs[4 * s + 1], segs[4 * s + 2], segs[4 * s + 3]);
        int4 L;
        snap(F.x, ds.S, L.x);
        snap(F.y, ds.S, L.y);
        snap(F.z, ds.S, L.z);
        snap(F.w, ds.S, L.w);
        seg_lat[s] = L;
        seg_pos[s] = F;
        const int g = np + 3 * s;  // A, B, interior (stored at A)
        gen_lat[g] = make_int2(L.x, L.y);
        gen_lat[g + 1] = make_int2(L.z, L.w);
        gen_lat[g + 2] = make_int2(L.x, L.y);
        gen_pos[g] = make_float2(F.x, F.y);
        gen_pos[g + 1] = make_float2(F.z, F.w);
        gen_pos[g + 2] = make_float2(F.x, F.y);
    }
}

}  // namespace

void launch_update_sources(const DevScene &ds, cudaStream_t st, const float *pts, const float *segs) {
    k_update_sources<<<1, kUpdThreads, 0, st>>>(ds, pts, segs);
}

}  // namespace spm
