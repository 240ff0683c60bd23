// spm_sequential.cu -- the paper's generator-sequential schedule (Sec. 3.1,
// Procedures 1-4) as one cooperative CUDA kernel: the A/B baseline for the
// culled gather of spm_compute. It computes the map the way the paper's
// shader pipeline does, one generator at a time over every pixel.
//
// Iteration k, every CTA of the grid:
//   Procedure 1 -- finds the unexpanded generator of least cost (ties: the
//     smaller id). All CTAs read the same state and so agree; each keeps its
//     own copy of the expanded flags in shared memory.
//   Procedure 4 -- every unexpanded obstacle vertex the generator sees
//     exactly takes cost(g) + |v - g| (FP64; the perpendicular distance for a
//     segment interior, Sec. 4) when that is smaller.
//   Procedures 2 + 3 -- every free pixel takes the packed (FP32 distance, id)
//     key of the generator when it is smaller than its own (the depth test)
//     and the generator is visible from it. The exact visibility test stands
//     in for the stencil of shadow triangles and runs only for pixels whose
//     depth test passes, as early depth testing does on the paper's GPU; the
//     result is the same.
// Vertex costs alternate between two buffers by iteration, so one grid
// barrier per iteration separates the reads of Procedure 1 from the writes
// of Procedure 4. The pixel keys live in the output planes themselves
// (distance, parent id), like the paper's framebuffer. Unlike spm_compute
// there are no shadow cones and no tangency filter: the paper has neither.
// The loop stops once no unexpanded generator has a finite cost (the
// remaining ones would change nothing).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "spm_device.cuh"
#include "spm_internal.h"

namespace spm {
namespace {

namespace cg = cooperative_groups;

constexpr int kSeqThreads = 256;
constexpr int kNonFree = -2;  // parent plane marker of a pixel inside an obstacle (until the end)

// Pixel centre (lattice) inside the open interior of an obstacle?
__device__ bool pixel_inside_obstacle(const DevScene &ds, int px, int py) {
    const int bx = (px - ds.bin_x0) / ds.bin_size, by = (py - ds.bin_y0) / ds.bin_size;
    if (bx < 0 || by < 0 || bx >= ds.bin_nx || by >= ds.bin_ny) return false;
    const int bin = by * ds.bin_nx + bx;
    for (int it = ds.bin_start[bin]; it < ds.bin_start[bin + 1]; ++it) {
        const BinRec rec = ds.bin_recs[it];
        if (px <= rec.box.x || px >= rec.box.z || py <= rec.box.y || py >= rec.box.w) continue;
        bool inside = true;
        for (int e = 0; e < rec.m && inside; ++e) {
            const int2 a = ds.poly_v[rec.voff + e], c = ds.poly_v[rec.voff + (e + 1 == rec.m ? 0 : e + 1)];
            inside = orient32(a.x, a.y, c.x, c.y, px, py) > 0;
        }
        if (inside) return true;
    }
    return false;
}

// FP64 length of the link from generator g to obstacle vertex v (correctly
// rounded operations; perpendicular distance for a segment interior).
__device__ __forceinline__ double link_len(const DevScene &ds, int kind, int g, float2 vp) {
    if (kind == kSegI) {
        const float4 F = ds.seg_pos[ds.gen_aux[g]];
        const double ux = __dsub_rn((double)F.z, (double)F.x), uy = __dsub_rn((double)F.w, (double)F.y);
        const double c = __dsub_rn(__dmul_rn(ux, __dsub_rn((double)vp.y, (double)F.y)),
                                   __dmul_rn(uy, __dsub_rn((double)vp.x, (double)F.x)));
        return __ddiv_rn(fabs(c), __dsqrt_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy))));
    }
    const float2 gp = ds.gen_pos[g];
    const double dx = __dsub_rn((double)vp.x, (double)gp.x), dy = __dsub_rn((double)vp.y, (double)gp.y);
    return __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

__global__ void __launch_bounds__(kSeqThreads) k_sequential(const __grid_constant__ DevScene ds,
                                                            float *__restrict__ dist,
                                                            int32_t *__restrict__ parent) {
    cg::grid_group grid = cg::this_grid();
    __shared__ uint32_t expanded[kSeqMaxGen / 32];
    __shared__ double wc[kSeqThreads / 32];
    __shared__ int wi[kSeqThreads / 32];
    const int n = ds.n_gen;
    const long long gtid = (long long)blockIdx.x * kSeqThreads + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * kSeqThreads;
    const long long npx = (long long)ds.Nx * ds.Ny;
    const int pitch_x = ds.S * ds.Wx / ds.Nx, pitch_y = ds.S * ds.Wy / ds.Ny;
    for (int w = threadIdx.x; w < (n + 31) / 32; w += kSeqThreads) expanded[w] = 0u;
    for (long long g = gtid; g < n; g += gthreads)
        for (int b = 0; b < 2; ++b) {
            ds.cost[b][g] = g < ds.n_src ? 0.0 : (double)INFINITY;
            ds.par[b][g] = g < ds.n_src ? (int)g : -1;
        }
    for (long long q = gtid; q < npx; q += gthreads) {
        const int i = (int)(q % ds.Nx), j = (int)(q / ds.Nx);
        dist[q] = INFINITY;
        parent[q] = pixel_inside_obstacle(ds, pitch_x * i + pitch_x / 2, pitch_y * j + pitch_y / 2) ? kNonFree : -1;
    }
    grid.sync();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int it = 0; it < n; ++it) {
        const double *cc = ds.cost[it & 1];
        const int32_t *pc = ds.par[it & 1];
        double *cn = ds.cost[(it + 1) & 1];
        int32_t *pn = ds.par[(it + 1) & 1];
        // Procedure 1: the unexpanded generator of least cost
        double bc = INFINITY;
        int bi = INT_MAX;
        for (int g = threadIdx.x; g < n; g += kSeqThreads) {
            if ((expanded[g >> 5] >> (g & 31)) & 1u) continue;
            const double c = __ldcg(cc + g);
            if (c < bc) {  // g grows along this thread's walk: equal costs keep the smaller id
                bc = c;
                bi = g;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double oc = __shfl_xor_sync(0xffffffffu, bc, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (oc < bc || (oc == bc && oi < bi)) {
                bc = oc;
                bi = oi;
            }
        }
        if (lane == 0) {
            wc[warp] = bc;
            wi[warp] = bi;
        }
        __syncthreads();
        bc = wc[0];
        bi = wi[0];
        for (int w = 1; w < kSeqThreads / 32; ++w)
            if (wc[w] < bc || (wc[w] == bc && wi[w] < bi)) {
                bc = wc[w];
                bi = wi[w];
            }
        __syncthreads();  // wc / wi are rewritten next iteration
        if (!(bc < (double)INFINITY)) break;  // every CTA reads the same state: all leave together
        const int g = bi;
        if (threadIdx.x == 0) expanded[g >> 5] |= 1u << (g & 31);
        const int kind = ds.gen_kind[g];
        const int2 gl = ds.gen_lat[g];
        const float2 gp = ds.gen_pos[g];
        const float cf = (float)bc;
        int4 L = make_int4(0, 0, 0, 0);
        float4 F = make_float4(0.f, 0.f, 0.f, 0.f);
        long long den = 1;
        float seg_il = 0.f;
        if (kind == kSegI) {
            L = ds.seg_lat[ds.gen_aux[g]];
            F = ds.seg_pos[ds.gen_aux[g]];
            den = (long long)(L.z - L.x) * (L.z - L.x) + (long long)(L.w - L.y) * (L.w - L.y);
            const float fux = F.z - F.x, fuy = F.w - F.y;
            seg_il = 1.0f / sqrtf(fux * fux + fuy * fuy);
        }
        // Procedure 4: obstacle vertices the generator sees
        for (long long v = ds.n_src + gtid; v < n; v += gthreads) {
            double c = __ldcg(cc + v);
            int p = __ldcg(pc + v);
            if (v != g && !((expanded[v >> 5] >> (v & 31)) & 1u)) {
                const int2 vl = ds.gen_lat[v];
                bool sees = false;
                if (kind == kSegI) {
                    const long long num = (long long)(vl.x - L.x) * (L.z - L.x) + (long long)(vl.y - L.y) * (L.w - L.y);
                    sees = num > 0 && num < den && visible_foot(ds, ds.gen_aux[g], vl.x, vl.y, num, den);
                } else {
                    sees = visible_points(ds, vl.x, vl.y, gl.x, gl.y);
                }
                if (sees) {
                    const double cand = __dadd_rn(bc, link_len(ds, kind, g, ds.gen_pos[v]));
                    if (cand < c) {
                        c = cand;
                        p = g;
                    }
                }
            }
            cn[v] = c;
            pn[v] = p;
        }
        // Procedures 2 + 3: the depth test, then exact visibility
        for (long long q = gtid; q < npx; q += gthreads) {
            const int cur_p = parent[q];
            if (cur_p == kNonFree) continue;
            const int i = (int)(q % ds.Nx), j = (int)(q / ds.Nx);
            const int px = pitch_x * i + pitch_x / 2, py = pitch_y * j + pitch_y / 2;
            const float fx = ((float)i + 0.5f) * ds.hx, fy = ((float)j + 0.5f) * ds.hy;
            float d;
            long long num = 0;
            if (kind == kSegI) {
                num = (long long)(px - L.x) * (L.z - L.x) + (long long)(py - L.y) * (L.w - L.y);
                if (!(num > 0 && num < den)) continue;
                d = fabsf((F.z - F.x) * (fy - F.y) - (F.w - F.y) * (fx - F.x)) * seg_il;
            } else {
                const float ddx = fx - gp.x, ddy = fy - gp.y;
                d = cf + sqrtf(ddx * ddx + ddy * ddy);
            }
            const unsigned long long kk = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)g;
            const unsigned long long cur = ((unsigned long long)__float_as_uint(dist[q]) << 32) | (unsigned)cur_p;
            if (kk >= cur) continue;
            const bool vis = kind == kSegI ? visible_foot(ds, ds.gen_aux[g], px, py, num, den)
                                           : visible_points(ds, px, py, gl.x, gl.y);
            if (vis) {
                dist[q] = d;
                parent[q] = g;
            }
        }
        grid.sync();
    }
    grid.sync();
    for (long long q = gtid; q < npx; q += gthreads)
        if (parent[q] == kNonFree) parent[q] = -1;
}

}  // namespace

int sequential_grid_blocks() {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sequential, kSeqThreads, 0);
    return (sms > 0 ? sms : 1) * (per_sm < 1 ? 1 : per_sm);
}

cudaError_t launch_sequential(const DevScene &ds, cudaStream_t st, float *dist, int32_t *parent, int blocks) {
    void *args[] = {(void *)&ds, (void *)&dist, (void *)&parent};
    return cudaLaunchCooperativeKernel((const void *)k_sequential, dim3(blocks), dim3(kSeqThreads), args, 0, st);
}

}  // namespace spm
