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

constexpr int kFloodWarps = 4;
constexpr int kFloodThreads = 32 * kFloodWarps;
constexpr int kQueue = 1024;  // per-warp ring buffer of tiles

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

__global__ void __launch_bounds__(kFloodThreads) k_flood(DevScene ds) {
    extern __shared__ unsigned fsm[];
    if (ds.flood_mode == 0) {  // automatic: flood only sparse visibility graphs
        const double pairs = (double)ds.n_gen * (double)max(ds.n_vert, 1);
        if ((double)ds.in_start[ds.n_vert] > 0.01 * pairs) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ds.flood_counts[2] = 1;
            return;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = ds.tiles_x * ds.tiles_y, words = (ntiles + 31) / 32;
    unsigned *visited = fsm + warp * (words + kQueue);
    int *queue = (int *)(visited + words);
    const int nwarps = gridDim.x * kFloodWarps;
    const int tpx = ds.tile * (ds.S * ds.Wx / ds.Nx), tpy = ds.tile * (ds.S * ds.Wy / ds.Ny);
    for (int g = blockIdx.x * kFloodWarps + warp; g < ds.n_gen; g += nwarps) {
        if (!(ds.gen_costf[g] < INFINITY)) continue;
        const int kind = ds.gen_kind[g];
        const int ct = kind == kVert ? ds.gen_ctype[g] : kConeNone;
        if (ct == kConeEmpty) continue;
        const int2 gl = ds.gen_lat[g];
        const int tx = gl.x >= 0 ? gl.x / tpx : -1, ty = gl.y >= 0 ? gl.y / tpy : -1;
        if (kind == kSegI) {
            if (lane == 0) push_global(ds, g);
            continue;
        }
        const int4 cone = kind == kVert ? ds.gen_cone[g] : make_int4(0, 0, 0, 0);
        for (int w = lane; w < words; w += 32) visited[w] = 0u;
        __syncwarp();
        // seeds: every tile whose closed area contains g (up to 4 when g lies
        // on tile edges)
        bool fresh = false;
        int t0 = 0;
        if (lane < 4) {
            const int sx = tx - (lane & 1), sy = ty - ((lane >> 1) & 1);
            if (tx >= 0 && ty >= 0 && sx >= 0 && sy >= 0 && sx < ds.tiles_x && sy < ds.tiles_y) {
                const int4 a4 = tile_area(ds, sx, sy);
                if (gl.x >= a4.x && gl.x <= a4.z && gl.y >= a4.y && gl.y <= a4.w) {
                    t0 = sy * ds.tiles_x + sx;
                    fresh = !(atomicOr(&visited[t0 >> 5], 1u << (t0 & 31)) & (1u << (t0 & 31)));
                }
            }
        }
        const unsigned sb = __ballot_sync(0xffffffffu, fresh);
        if (fresh) queue[__popc(sb & ((1u << lane) - 1u))] = t0;
        int head = 0, tail = __popc(sb);
        if (tail == 0) {  // g outside every tile: scanned by all tiles instead
            if (lane == 0) push_global(ds, g);
            continue;
        }
        bool overflow = false;
        while (head < tail && !overflow) {
            // the whole warp tests one frontier tile (uniform control flow)
            const int t = queue[head % kQueue];
            ++head;
            const int cx = t % ds.tiles_x, cy = t / ds.tiles_x;
            const int4 area = tile_area(ds, cx, cy);
            bool ok = cone_meets_box(ct, cone, gl, area);
            if (ok) {
                const float acx = 0.5f * ((float)area.x + (float)area.z), acy = 0.5f * ((float)area.y + (float)area.w);
                const float ar = 0.5f * sqrtf((float)(area.z - area.x) * (float)(area.z - area.x) +
                                              (float)(area.w - area.y) * (float)(area.w - area.y)) + 1.0f;
                ok = !box_hidden_warp(ds, gl, area, acx, acy, ar);
                if (lane == 0) {
                    SPM_CNT(11, 1);
                    SPM_CNT(12, ok ? 1 : 0);
                }
            }
            if (!ok) continue;
            if (lane == 0) {  // emit (tile, g)
                const int slot = atomicAdd(&ds.flood_counts[0], 1);
                if (slot < ds.pair_cap) {
                    ds.pairs[slot] = make_int2(t, g);
                    atomicAdd(&ds.tile_count[t], 1);
                } else {
                    atomicOr(&ds.flood_counts[2], 1);
                }
            }
            // lanes 0..8 look at the 8-neighbours, fresh ones join the queue
            bool nfresh = false;
            int nt = 0;
            if (lane < 9 && lane != 4) {
                const int nx = cx + lane % 3 - 1, ny = cy + lane / 3 - 1;
                if (nx >= 0 && ny >= 0 && nx < ds.tiles_x && ny < ds.tiles_y) {
                    nt = ny * ds.tiles_x + nx;
                    nfresh = !(atomicOr(&visited[nt >> 5], 1u << (nt & 31)) & (1u << (nt & 31)));
                }
            }
            const unsigned pb = __ballot_sync(0xffffffffu, nfresh);
            if (nfresh) queue[(tail + __popc(pb & ((1u << lane) - 1u))) % kQueue] = nt;
            tail += __popc(pb);
            if (tail - head > kQueue) overflow = true;
        }
        if (overflow && lane == 0) {
            push_global(ds, g);
            SPM_CNT(13, 1);
        }
        __syncwarp();
    }
}

// Exclusive scan of tile_count into tile_start (one CTA), then fill.
__global__ void __launch_bounds__(1024) k_tiles_scan(DevScene ds) {
    __shared__ long long part[1024];
    const int n = ds.tiles_x * ds.tiles_y;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(n, lo + per);
    long long s = 0;
    for (int i = lo; i < hi; ++i) s += ds.tile_count[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            long long x = part[t];
            part[t] = run;
            run += x;
        }
    }
    __syncthreads();
    long long run = part[threadIdx.x];
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

size_t flood_smem_bytes(int tiles) {
    const int words = (tiles + 31) / 32;
    return sizeof(unsigned) * (size_t)kFloodWarps * (words + kQueue);
}

bool flood_possible(int tiles) { return flood_smem_bytes(tiles) <= 200 * 1024; }

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
    const int blocks = min(152 * 8, (ds.n_gen + kFloodWarps - 1) / kFloodWarps);
    k_flood<<<max(blocks, 1), kFloodThreads, smem, st>>>(ds);
    k_tiles_scan<<<1, 1024, 0, st>>>(ds);
    k_tiles_fill<<<152 * 4, 256, 0, st>>>(ds);
}

int flood_smem_attr() {
    return cudaFuncSetAttribute(k_flood, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) == cudaSuccess;
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
