// spm_flood.cu -- per-tile candidate lists by flooding each generator's
// potentially visible tiles (the per-tile culling step of the pixel pass).
//
// For a point generator g (point source, segment endpoint, obstacle vertex),
// the pixels that see g and lie in its shadow cone form a region that is
// star-shaped from g: the segment from g to any such pixel stays inside the
// cone and sees g all along. Every tile that segment crosses therefore holds
// visible points. A breadth-first flood over tiles from g's tile, expanding a
// tile only when it meets the cone and is not hidden from g by a single
// polygon between it and g, thus reaches every tile where g can win (tiles are closed
// rectangles that tile the plane; 8-neighbour steps follow any segment).
// Each reached tile gets g in its candidate list. Segment interiors, points
// outside the tile grid and floods that outgrow their queue go to a global
// list that every tile scans. Any failure of the lists (pair capacity) sets a
// flag and the pixel pass falls back to scanning every generator.
#include <cuda_runtime.h>

#include "spm_device.cuh"
#include "spm_internal.h"

namespace spm {
namespace {

constexpr int kFloodThreads = 256;  // one CTA floods one generator at a time
constexpr int kFront = 1024;        // frontier tiles per breadth-first level

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

// The bins that can hold a polygon hiding a tile from g: the thick segment
// from the tile centre c to g (radius r, the tile's half diagonal + 1), cut
// into strips of bins along its major axis. Each strip is one work item.
struct StripWalk {
    float pu, pw, du, dw, ou, ow, m;
    int us, ustep, nstrips, nw;
    bool xmaj;
};

__device__ __forceinline__ int bin_clamp(float v, float o, float bs, int n) {
    const int b = (int)floorf((v - o) / bs);
    return b < 0 ? 0 : (b >= n ? n - 1 : b);
}

__device__ __forceinline__ StripWalk strip_walk(const DevScene &ds, int2 g, float cx, float cy, float r) {
    StripWalk w;
    const float tx = (float)g.x, ty = (float)g.y, bs = (float)ds.bin_size;
    w.m = r + 1.0f;
    w.xmaj = fabsf(tx - cx) >= fabsf(ty - cy);
    w.pu = w.xmaj ? cx : cy;
    w.pw = w.xmaj ? cy : cx;
    const float qu = w.xmaj ? tx : ty, qw = w.xmaj ? ty : tx;
    w.ou = w.xmaj ? (float)ds.bin_x0 : (float)ds.bin_y0;
    w.ow = w.xmaj ? (float)ds.bin_y0 : (float)ds.bin_x0;
    const int nu = w.xmaj ? ds.bin_nx : ds.bin_ny;
    w.nw = w.xmaj ? ds.bin_ny : ds.bin_nx;
    const int u0 = bin_clamp(fminf(w.pu, qu) - w.m, w.ou, bs, nu), u1 = bin_clamp(fmaxf(w.pu, qu) + w.m, w.ou, bs, nu);
    w.ustep = qu >= w.pu ? 1 : -1;
    w.us = w.ustep > 0 ? u0 : u1;
    w.nstrips = u1 - u0 + 1;
    w.du = qu - w.pu;
    w.dw = qw - w.pw;
    return w;
}

// Upper bound on the bins one strip spans across the minor axis: the strip's
// major-axis extent is bs + 2m, the segment moves |dw/du| per unit along it,
// and the span grows by m on both sides.
__device__ __forceinline__ int strip_bins_max(const DevScene &ds, const StripWalk &w) {
    const float bs = (float)ds.bin_size;
    const float slope = fabsf(w.du) < 0.5f ? 0.f : fabsf(w.dw / w.du);
    const float span = fabsf(w.du) < 0.5f ? fabsf(w.dw) + 2.f * w.m : slope * (bs + 2.f * w.m) + 2.f * w.m;
    return min((int)(span / bs) + 2, w.nw);
}

// Does one polygon in bin k of strip sidx hide every point of box from g?
// Stops early once another item has found a hiding polygon for the same tile.
__device__ __forceinline__ bool bin_hides(const DevScene &ds, const StripWalk &w, int sidx, int k, int2 g, int4 box, float cx,
                          float cy, float r, const volatile int *stop) {
    const float bs = (float)ds.bin_size;
    const int u = w.us + w.ustep * sidx;
    float wlo, whi;
    if (fabsf(w.du) < 0.5f) {
        wlo = fminf(w.pw, w.pw + w.dw);
        whi = fmaxf(w.pw, w.pw + w.dw);
    } else {
        const float a = w.ou + u * bs - w.m, b = w.ou + (u + 1) * bs + w.m;
        const float t0 = (a - w.pu) / w.du, t1 = (b - w.pu) / w.du;
        float tl = fmaxf(0.f, fminf(t0, t1)), th = fminf(1.f, fmaxf(t0, t1));
        if (tl > th) { tl = 0.f; th = 1.f; }
        const float wa = w.pw + tl * w.dw, wb = w.pw + th * w.dw;
        wlo = fminf(wa, wb);
        whi = fmaxf(wa, wb);
    }
    const int v = bin_clamp(wlo - w.m, w.ow, bs, w.nw) + k;
    if (v > bin_clamp(whi + w.m, w.ow, bs, w.nw)) return false;
    const float tx = (float)g.x, ty = (float)g.y;
    const int bin = w.xmaj ? v * ds.bin_nx + u : u * ds.bin_nx + v;
    const int e = __ldg(ds.bin_start + bin + 1);
    for (int it = __ldg(ds.bin_start + bin); it < e; ++it) {
        if (*stop) return false;
        const int4 *rp = reinterpret_cast<const int4 *>(ds.bin_recs + it);
        const int4 rbox = __ldg(rp), rmeta = __ldg(rp + 1);  // box; poly, voff, m
        if (!seg_near_box(cx, cy, tx, ty, r, rbox)) continue;
        const int2 *V = ds.poly_v + rmeta.y;
        const int m = rmeta.z;
        const unsigned mg = edge_mask(V, m, g.x, g.y);
        if (poly_blocks(V, m, box.x, box.y, g.x, g.y, mg) && poly_blocks(V, m, box.z, box.y, g.x, g.y, mg) &&
            poly_blocks(V, m, box.x, box.w, g.x, g.y, mg) && poly_blocks(V, m, box.z, box.w, g.x, g.y, mg))
            return true;
    }
    return false;
}

struct FloodSmem {
    int front[2][kFront];  // current / next breadth-first level
    int pre[kFront + 1];   // exclusive prefix of (strip, bin) items per frontier tile
    int flag[kFront];      // 0 visible, 1 hidden, 2 outside the cone
    int cnt[2];
    int overflow;
    int wsum[kFloodThreads / 32];
};

// Exclusive scan of v[0..n) in place (n <= kFront), v[n] = total. All threads.
__device__ void cta_scan(int *v, int n, int *wsum) {
    constexpr int per = (kFront + kFloodThreads - 1) / kFloodThreads;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int loc[per];
    int s = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int i = threadIdx.x * per + k;
        loc[k] = i < n ? v[i] : 0;
        s += loc[k];
    }
    int inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    int run = inc - s;
    for (int w = 0; w < warp; ++w) run += wsum[w];
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int i = threadIdx.x * per + k;
        if (i < n) v[i] = run;
        run += loc[k];
    }
    if (threadIdx.x == kFloodThreads - 1) v[n] = run;
}

__global__ void __launch_bounds__(kFloodThreads) k_flood(DevScene ds) {
    extern __shared__ unsigned visited[];
    __shared__ FloodSmem sm;
    if (ds.flood_mode == 0) {  // automatic: flood only sparse visibility graphs
        const double pairs = (double)ds.n_gen * (double)max(ds.n_vert, 1);
        if ((double)ds.in_start[ds.n_vert] > 0.01 * pairs) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ds.flood_counts[2] = 1;
            return;
        }
    }
    const int tid = threadIdx.x;
    const int ntiles = ds.tiles_x * ds.tiles_y, words = (ntiles + 31) / 32;
    const int tpx = ds.tile * (ds.S * ds.Wx / ds.Nx), tpy = ds.tile * (ds.S * ds.Wy / ds.Ny);
    for (int g = blockIdx.x; g < ds.n_gen; g += gridDim.x) {
        if (!(ds.gen_costf[g] < INFINITY)) continue;
        const int kind = ds.gen_kind[g];
        const int ct = kind == kVert ? ds.gen_ctype[g] : kConeNone;
        if (ct == kConeEmpty) continue;
        if (kind == kSegI) {
            if (tid == 0) push_global(ds, g);
            continue;
        }
        const int2 gl = ds.gen_lat[g];
        const int4 cone = kind == kVert ? ds.gen_cone[g] : make_int4(0, 0, 0, 0);
        const int tx = gl.x >= 0 ? gl.x / tpx : -1, ty = gl.y >= 0 ? gl.y / tpy : -1;
        __syncthreads();  // the previous generator's last level is done with smem
        for (int w = tid; w < words; w += kFloodThreads) visited[w] = 0u;
        if (tid == 0) {
            sm.cnt[0] = 0;
            sm.overflow = 0;
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
        if (sm.cnt[0] == 0) {  // g outside every tile: scanned by all tiles instead
            if (tid == 0) push_global(ds, g);
            continue;
        }
#ifdef SPM_COUNT
        int n_tests = 0;
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
            // A: cone test and strip count per frontier tile
            for (int i = tid; i < nc; i += kFloodThreads) {
                const int t = cur[i];
                const int4 area = tile_area(ds, t % ds.tiles_x, t / ds.tiles_x);
                const bool ok = cone_meets_box(ct, cone, gl, area);
                int ns = 0;
                if (ok) {
                    const float acx = 0.5f * ((float)area.x + (float)area.z), acy = 0.5f * ((float)area.y + (float)area.w);
                    const float ar = 0.5f * sqrtf((float)(area.z - area.x) * (float)(area.z - area.x) +
                                                  (float)(area.w - area.y) * (float)(area.w - area.y)) + 1.0f;
                    const StripWalk w = strip_walk(ds, gl, acx, acy, ar);
                    ns = w.nstrips * strip_bins_max(ds, w);
                }
                sm.flag[i] = ok ? 0 : 2;
                sm.pre[i] = ns;
            }
            if (tid == 0) sm.cnt[p ^ 1] = 0;
            __syncthreads();
            cta_scan(sm.pre, nc, sm.wsum);
            __syncthreads();
            // B: every (tile, strip, bin) item in parallel; a hiding polygon sets the tile's flag
            const int total = sm.pre[nc];
            for (int j = tid; j < total; j += kFloodThreads) {
                int lo = 0, hi = nc;  // pre[lo] <= j < pre[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (sm.pre[mid] <= j) lo = mid;
                    else hi = mid;
                }
                volatile int *fl = &sm.flag[lo];
                if (*fl) continue;
                const int t = cur[lo];
                const int4 area = tile_area(ds, t % ds.tiles_x, t / ds.tiles_x);
                const float acx = 0.5f * ((float)area.x + (float)area.z), acy = 0.5f * ((float)area.y + (float)area.w);
                const float ar = 0.5f * sqrtf((float)(area.z - area.x) * (float)(area.z - area.x) +
                                              (float)(area.w - area.y) * (float)(area.w - area.y)) + 1.0f;
                const StripWalk w = strip_walk(ds, gl, acx, acy, ar);
                const int kb = strip_bins_max(ds, w), q = j - sm.pre[lo];
                if (bin_hides(ds, w, q / kb, q - (q / kb) * kb, gl, area, acx, acy, ar, fl)) *fl = 1;
            }
            __syncthreads();
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
            if (tid == 0)
                for (int i = 0; i < nc; ++i) n_tests += sm.flag[i] != 2;
#endif
            __syncthreads();
            p ^= 1;
        }
#ifdef SPM_COUNT
        if (tid == 0) {
            SPM_CNT_MAX(14, n_tests);
            SPM_CNT(15, n_tests > 256 ? 1 : 0);
        }
#endif
    }
}

// Exclusive scan of tile_count into tile_start (one CTA), then fill.
__global__ void __launch_bounds__(1024) k_tiles_scan(DevScene ds) {
    __shared__ long long wsum[32];
    const int n = ds.tiles_x * ds.tiles_y;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(n, lo + per);
    long long s = 0;
    for (int i = lo; i < hi; ++i) s += ds.tile_count[i];
    long long run = cta_exclusive_scan(s, wsum);
    for (int i = lo; i < hi; ++i) {
        ds.tile_start[i] = (int32_t)run;
        run += ds.tile_count[i];
        ds.tile_count[i] = 0;  // reused as fill cursor
    }
    if (hi == n && lo < hi) ds.tile_start[n] = (int32_t)run;
    if (threadIdx.x == 0 && n == 0) ds.tile_start[0] = 0;
}

__global__ void k_tiles_fill(DevScene ds) {
    const int np = min(ds.flood_counts[0], ds.pair_cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const int2 pr = ds.pairs[i];
        const int slot = atomicAdd(&ds.tile_count[pr.x], 1);
        ds.tile_items[ds.tile_start[pr.x] + slot] = pr.y;
    }
}

}  // namespace

size_t flood_smem_bytes(int tiles) {  // dynamic part: the visited bitmap
    return sizeof(unsigned) * (size_t)((tiles + 31) / 32);
}

bool flood_possible(int tiles) { return flood_smem_bytes(tiles) + sizeof(FloodSmem) <= 200 * 1024; }

void launch_flood(const DevScene &ds, cudaStream_t st) {
    const int ntiles = ds.tiles_x * ds.tiles_y;
    if (ds.flood_mode == 2) {  // never: the pixel pass scans every generator
        static const int32_t off[4] = {0, 0, 1, 0};
        cudaMemcpyAsync(ds.flood_counts, off, sizeof off, cudaMemcpyHostToDevice, st);
        return;
    }
    cudaMemsetAsync(ds.tile_count, 0, sizeof(int32_t) * ntiles, st);
    cudaMemsetAsync(ds.flood_counts, 0, sizeof(int32_t) * 4, st);
    const size_t smem = flood_smem_bytes(ntiles);
    const int blocks = min(152 * 4, ds.n_gen);
    k_flood<<<max(blocks, 1), kFloodThreads, smem, st>>>(ds);
    k_tiles_scan<<<1, 1024, 0, st>>>(ds);
    k_tiles_fill<<<152 * 4, 256, 0, st>>>(ds);
}

int flood_smem_attr() {
    return cudaFuncSetAttribute(k_flood, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024 - (int)sizeof(FloodSmem)) == cudaSuccess;
}

}  // namespace spm

#ifdef SPM_COUNT
// Instrumentation build only: reads and clears this unit's work counters.
extern "C" int spm_debug_counters_flood(unsigned long long *out16) {
    cudaDeviceSynchronize();
    if (cudaMemcpyFromSymbol(out16, spm::g_count, sizeof(unsigned long long) * 16) != cudaSuccess) return 1;
    unsigned long long z[16] = {0};
    cudaMemcpyToSymbol(spm::g_count, z, sizeof z);
    return 0;
}
#endif
