// spm_vertex.cu -- vertex phase: costs of obstacle-vertex generators.
//
// arxiv 1805.08500 Sec. 3.1 settles generators one at a time (Procedure 1
// picks the minimum unexpanded entry, Procedure 4 relaxes every vertex that
// sees it). Here the same costs are reached as the fixpoint of
//     cost(v) = min over generators u that see v, with v inside u's shadow
//               cone, of cost(u) + |u - v|
// computed on the GPU in three steps:
//   1. k_vis_pairs: one bit per (generator u, obstacle vertex v) pair, set when
//      u sees v exactly and the line uv is tangent to u's obstacle wedge (a
//      vertex can only pass a path on along a tangent, so other pairs can never
//      relax v); segment interiors reach v through its perpendicular foot.
//   2. k_edges_*: the bits become CSR in-lists (by v) with FP64 edge lengths
//      and out-lists (by u) for frontier marking.
//   3. k_sssp: one CTA runs Jacobi rounds restricted to the frontier until no
//      cost or parent changes (bounded round count -> status bit).
// Costs are FP64 with explicitly rounded operations, so they match a plain
// FP64 Dijkstra over the same edges bit for bit.
#include <cuda_runtime.h>

#include "spm_device.cuh"
#include "spm_internal.h"

namespace spm {
namespace {

constexpr int kVisThreads = 256;
constexpr int kSsspThreads = 1024;

// Static filter + exact visibility for one (u, v) pair.
__device__ bool pair_edge(const DevScene &ds, int u, int v) {
    if (u == v) return false;
    const int ku = ds.gen_kind[u];
    const int2 vl = ds.gen_lat[v];
    if (ku == kSegI) {
        int4 L = ds.seg_lat[ds.gen_aux[u]];
        long long ux = L.z - L.x, uy = L.w - L.y;
        long long num = (vl.x - L.x) * ux + (vl.y - L.y) * uy;
        long long den = ux * ux + uy * uy;
        if (!(num > 0 && num < den)) return false;
        return visible_foot(ds, ds.gen_aux[u], vl.x, vl.y, num, den);
    }
    const int2 ul = ds.gen_lat[u];
    if (ul.x == vl.x && ul.y == vl.y) return false;
    if (ku == kVert) {  // tangent at u: the line uv does not split u's wedge
        int4 w = ds.gen_wedge[u];
        int wx = vl.x - ul.x, wy = vl.y - ul.y;
        int a = cross32(wx, wy, w.x, w.y), b = cross32(wx, wy, w.z, w.w);
        if ((a > 0 && b < 0) || (a < 0 && b > 0)) return false;
    }
    return visible_points(ds, vl.x, vl.y, ul.x, ul.y);
}

// Row v (vertex index) of the bit matrix, word w covers generators 32w..32w+31.
__global__ void __launch_bounds__(kVisThreads) k_vis_pairs(DevScene ds) {
    const int lane = threadIdx.x & 31;
    const long long tasks = (long long)ds.n_vert * ds.vis_words;
    const long long warps = (long long)gridDim.x * (kVisThreads / 32);
    for (long long t = (long long)blockIdx.x * (kVisThreads / 32) + (threadIdx.x >> 5); t < tasks;
         t += warps) {
        const int vv = (int)(t / ds.vis_words), w = (int)(t % ds.vis_words);
        const int u = w * 32 + lane, v = ds.n_src + vv;
        bool e = (u < ds.n_gen) && pair_edge(ds, u, v);
        unsigned bits = __ballot_sync(0xffffffffu, e);
        if (lane == 0) ds.vis_bits[(size_t)vv * ds.vis_words + w] = bits;
    }
}

// In-degree per vertex row and out-degree per generator.
__global__ void k_edges_count(DevScene ds) {
    for (int vv = blockIdx.x * blockDim.x + threadIdx.x; vv < ds.n_vert; vv += gridDim.x * blockDim.x) {
        const uint32_t *row = ds.vis_bits + (size_t)vv * ds.vis_words;
        int cnt = 0;
        for (int w = 0; w < ds.vis_words; ++w) {
            uint32_t b = row[w];
            cnt += __popc(b);
            while (b) {
                int bit = __ffs(b) - 1;
                b &= b - 1;
                atomicAdd(&ds.out_start[w * 32 + bit + 1], 1);
            }
        }
        ds.in_start[vv + 1] = cnt;
    }
}

// Exclusive scans of in_start (n_vert + 1) and out_start (n_gen + 1), one CTA.
__global__ void __launch_bounds__(1024) k_edges_scan(DevScene ds) {
    __shared__ long long part[1024];
    for (int which = 0; which < 2; ++which) {
        int32_t *a = which == 0 ? ds.in_start : ds.out_start;
        const int n = which == 0 ? ds.n_vert : ds.n_gen;  // entries 1..n hold counts
        const int per = (n + blockDim.x - 1) / blockDim.x;
        const int lo = 1 + threadIdx.x * per, hi = min(n + 1, lo + per);
        long long s = 0;
        for (int i = lo; i < hi; ++i) s += a[i];
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

__global__ void k_edges_fill(DevScene ds) {
    if (ds.in_start[ds.n_vert] > ds.edge_cap) return;
    for (int vv = blockIdx.x * blockDim.x + threadIdx.x; vv < ds.n_vert; vv += gridDim.x * blockDim.x) {
        const uint32_t *row = ds.vis_bits + (size_t)vv * ds.vis_words;
        int e = ds.in_start[vv];
        const int v = ds.n_src + vv;
        for (int w = 0; w < ds.vis_words; ++w) {
            uint32_t b = row[w];
            while (b) {
                int u = w * 32 + __ffs(b) - 1;
                b &= b - 1;
                ds.in_src[e] = u;
                ds.in_len[e] = edge_len(ds, u, v);
                ++e;
                int slot = atomicAdd(&ds.out_fill[u], 1);
                ds.out_dst[ds.out_start[u] + slot] = v;
            }
        }
    }
}

// Jacobi rounds over the frontier in one CTA. cost[0]/par[0] hold the
// committed state; cost[1]/par[1] the values computed this round.
__global__ void __launch_bounds__(kSsspThreads) k_sssp(DevScene ds, int max_rounds) {
    extern __shared__ uint32_t dirty[];
    __shared__ int next_count, cur_count;
    const int n = ds.n_gen, nwords = (n + 31) / 32;
    if (ds.in_start[ds.n_vert] > ds.edge_cap) {
        if (threadIdx.x == 0) ds.stats[0] = 0;
        return;
    }
    double *cost = ds.cost[0], *ncost = ds.cost[1];
    int32_t *par = ds.par[0], *npar = ds.par[1];
    for (int g = threadIdx.x; g < n; g += blockDim.x) {
        const bool src = g < ds.n_src;
        cost[g] = src ? 0.0 : __longlong_as_double(0x7ff0000000000000ll);
        par[g] = src ? g : -1;
        if (src) ds.frontier[0][g] = g;
    }
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) dirty[w] = 0u;
    if (threadIdx.x == 0) { cur_count = ds.n_src; next_count = 0; }
    __syncthreads();
    int round = 0, fsel = 0;
    while (true) {
        const int *front = ds.frontier[fsel];
        int *nfront = ds.frontier[fsel ^ 1];
        const int fc = cur_count;
        if (fc == 0) break;
        if (round >= max_rounds) {
            if (threadIdx.x == 0) atomicOr(ds.status, kStNotConverged);
            break;
        }
        // mark out-neighbours of the frontier
        for (int i = threadIdx.x; i < fc; i += blockDim.x) {
            const int u = front[i];
            for (int e = ds.out_start[u]; e < ds.out_start[u + 1]; ++e) {
                const int v = ds.out_dst[e];
                atomicOr(&dirty[v >> 5], 1u << (v & 31));
            }
        }
        __syncthreads();
        // pull the dirty vertices from the committed state
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
            uint32_t b = dirty[w];
            dirty[w] = 0u;
            while (b) {
                const int v = w * 32 + __ffs(b) - 1;
                b &= b - 1;
                const int vv = v - ds.n_src;
                const int2 vl = ds.gen_lat[v];
                double best = __longlong_as_double(0x7ff0000000000000ll);
                int bpar = -1;
                for (int e = ds.in_start[vv]; e < ds.in_start[vv + 1]; ++e) {
                    const int u = ds.in_src[e];
                    const double cu = cost[u];
                    if (!(cu < best)) continue;  // cannot improve (edge lengths > 0)
                    if (ds.gen_kind[u] == kVert) {
                        int dx, dy;
                        arrival_dir(ds, par[u], ds.gen_lat[u], dx, dy);
                        int4 c;
                        int ct = make_cone(ds.gen_wedge[u], dx, dy, c);
                        const int2 ul = ds.gen_lat[u];
                        if (!in_cone(ct, c, vl.x - ul.x, vl.y - ul.y)) continue;
                    }
                    const double cand = __dadd_rn(cu, ds.in_len[e]);
                    if (cand < best || (cand == best && u < bpar)) {
                        best = cand;
                        bpar = u;
                    }
                }
                if (best != cost[v] || bpar != par[v]) {
                    ncost[v] = best;
                    npar[v] = bpar;
                    nfront[atomicAdd(&next_count, 1)] = v;
                }
            }
        }
        __syncthreads();
        const int nc = next_count;
        for (int i = threadIdx.x; i < nc; i += blockDim.x) {
            const int v = nfront[i];
            cost[v] = ncost[v];
            par[v] = npar[v];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            cur_count = nc;
            next_count = 0;
        }
        fsel ^= 1;
        ++round;
        __syncthreads();
    }
    if (threadIdx.x == 0) ds.stats[0] = round;
}

// Final generator table for the pixel phase: FP32 costs and shadow cones.
__global__ void k_finalize(DevScene ds) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ds.n_gen; g += gridDim.x * blockDim.x) {
        const double c = ds.cost[0][g];
        const int p = ds.par[0][g];
        ds.gen_cost[g] = c;
        ds.gen_par[g] = p;
        ds.gen_costf[g] = (float)c;
        int4 cone = make_int4(0, 0, 0, 0);
        int ct = kConeNone;
        if (g >= ds.n_src) {
            if (p < 0) {
                ct = kConeEmpty;
            } else {
                int dx, dy;
                arrival_dir(ds, p, ds.gen_lat[g], dx, dy);
                ct = make_cone(ds.gen_wedge[g], dx, dy, cone);
            }
        }
        ds.gen_cone[g] = cone;
        ds.gen_ctype[g] = ct;
    }
}

}  // namespace

void launch_vertex_phase(const DevScene &ds, cudaStream_t st) {
    cudaMemsetAsync(ds.out_start, 0, sizeof(int32_t) * (ds.n_gen + 1), st);
    cudaMemsetAsync(ds.out_fill, 0, sizeof(int32_t) * ds.n_gen, st);
    if (ds.n_vert > 0) {
        const long long tasks = (long long)ds.n_vert * ds.vis_words;
        long long blocks = (tasks + (kVisThreads / 32) - 1) / (kVisThreads / 32);
        blocks = blocks > 152 * 16 ? 152 * 16 : blocks;
        k_vis_pairs<<<(int)blocks, kVisThreads, 0, st>>>(ds);
        int eb = (ds.n_vert + 255) / 256;
        k_edges_count<<<eb, 256, 0, st>>>(ds);
        k_edges_scan<<<1, 1024, 0, st>>>(ds);
        k_edges_fill<<<eb, 256, 0, st>>>(ds);
    } else {
        cudaMemsetAsync(ds.in_start, 0, sizeof(int32_t) * (ds.n_vert + 1), st);
    }
    const size_t smem = sizeof(uint32_t) * ((ds.n_gen + 31) / 32);
    k_sssp<<<1, kSsspThreads, smem, st>>>(ds, 4 * ds.n_gen + 64);
    k_finalize<<<(ds.n_gen + 255) / 256, 256, 0, st>>>(ds);
}

int count_kernel_launches_vertex() { return 6; }

}  // namespace spm
