// spm_grad.cu -- differentiable form: agent loss and its adjoint.
//
// loss = (1/n) * sum over agents a of lambda*(a) (the field value at the
// agent's pixel; unreached agents contribute 0). lambda*(a) is the length of
// the parent chain a -> v_k -> ... -> root source (arxiv 1805.08500 Sec. 3.1,
// ParentId). Obstacle vertices do not move, so only the root link depends on
// the sources: with x the last point before the root,
//   point source s (or segment endpoint):  d lambda / d s = (s - x) / |s - x|
//   segment interior A->B, foot parameter t, unit normal n from foot to x:
//                                          d lambda / d A = -(1 - t) n,
//                                          d lambda / d B = -t n.
// All reductions run in a fixed order in FP64, so results are deterministic.
#include <cuda_runtime.h>

#include "spm_device.cuh"
#include "spm_internal.h"

namespace spm {
namespace {

// Root generator and last pre-root point for every generator's chain.
__global__ void k_root_table(DevScene ds, int32_t *root, float2 *lastpt) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ds.n_gen; g += gridDim.x * blockDim.x) {
        int r = g, guard = 0;
        float2 x = make_float2(0.f, 0.f);
        while (r >= 0 && ds.gen_kind[r] == kVert) {
            x = ds.gen_pos[r];
            r = ds.gen_par[r];
            if (++guard > ds.n_gen) { r = -1; break; }
        }
        root[g] = r;
        lastpt[g] = x;
    }
}

__global__ void __launch_bounds__(1024) k_loss(const int32_t *agents, int n, int Nx, int Ny,
                                               const float *dist, float *loss) {
    __shared__ double part[1024];
    double s = 0.0;
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
        const int i = agents[2 * a], j = agents[2 * a + 1];
        if (i < 0 || j < 0 || i >= Nx || j >= Ny) continue;
        const float d = dist[(size_t)j * Nx + i];
        if (d < INFINITY) s += (double)d;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(part[0] / (double)max(n, 1));
}

// Per-agent contribution: output slot base and up to four values.
__global__ void k_agent_contrib(DevScene ds, const int32_t *agents, int n, const int32_t *parent,
                                const int32_t *root, const float2 *lastpt, int32_t *slot,
                                float4 *val) {
    const int npt2 = 2 * (ds.n_src - 3 * ds.n_seg);
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        slot[a] = -1;
        val[a] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int i = agents[2 * a], j = agents[2 * a + 1];
        if (i < 0 || j < 0 || i >= ds.Nx || j >= ds.Ny) continue;
        const int g = parent[(size_t)j * ds.Nx + i];
        if (g < 0) continue;
        int r;
        float2 x;
        if (ds.gen_kind[g] == kVert) {
            r = root[g];
            x = lastpt[g];
            if (r < 0) continue;
        } else {
            r = g;
            x = make_float2(((float)i + 0.5f) * ds.hx, ((float)j + 0.5f) * ds.hy);
        }
        const int kind = ds.gen_kind[r], aux = ds.gen_aux[r];
        if (kind == kSegI) {
            const float4 F = ds.seg_pos[aux];
            const float ux = F.z - F.x, uy = F.w - F.y;
            const float t = ((x.x - F.x) * ux + (x.y - F.y) * uy) / (ux * ux + uy * uy);
            const float fx = F.x + t * ux, fy = F.y + t * uy;
            const float nx = x.x - fx, ny = x.y - fy, nn = sqrtf(nx * nx + ny * ny);
            if (!(nn > 0.f)) continue;
            const float ex = nx / nn, ey = ny / nn;
            slot[a] = npt2 + 4 * aux;
            val[a] = make_float4(-(1.f - t) * ex, -(1.f - t) * ey, -t * ex, -t * ey);
        } else {
            const float2 s = ds.gen_pos[r];
            const float dx = s.x - x.x, dy = s.y - x.y, nn = sqrtf(dx * dx + dy * dy);
            if (!(nn > 0.f)) continue;
            slot[a] = kind == kPoint ? 2 * aux : npt2 + 4 * aux + (kind == kSegB ? 2 : 0);
            val[a] = make_float4(dx / nn, dy / nn, 0.f, 0.f);
        }
    }
}

// One CTA per output component, fixed summation order.
__global__ void __launch_bounds__(256) k_agent_reduce(const int32_t *slot, const float4 *val, int n,
                                                      int n_pt2, float *grad_pts, float *grad_segs) {
    __shared__ double part[256];
    const int o = blockIdx.x;
    double s = 0.0;
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
        const int d = o - slot[a];
        if (slot[a] < 0 || d < 0 || d > 3) continue;
        const float4 v = val[a];
        s += (double)(d == 0 ? v.x : d == 1 ? v.y : d == 2 ? v.z : v.w);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) part[threadIdx.x] += part[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float g = (float)(part[0] / (double)max(n, 1));
        if (o < n_pt2) grad_pts[o] = g;
        else grad_segs[o - n_pt2] = g;
    }
}

}  // namespace

void launch_agents_forward(const DevScene &ds, cudaStream_t st, const int32_t *agents, int n,
                           const float *dist, float *loss) {
    k_loss<<<1, 1024, 0, st>>>(agents, n, ds.Nx, ds.Ny, dist, loss);
}

void launch_agents_backward(const DevScene &ds, cudaStream_t st, const int32_t *agents, int n,
                            const int32_t *parent, int32_t *root, float2 *lastpt, int32_t *slot,
                            float4 *val, float *grad_pts, float *grad_segs) {
    k_root_table<<<(ds.n_gen + 255) / 256, 256, 0, st>>>(ds, root, lastpt);
    const int blocks = n > 0 ? min((n + 255) / 256, 152 * 8) : 1;
    k_agent_contrib<<<blocks, 256, 0, st>>>(ds, agents, n, parent, root, lastpt, slot, val);
    const int n_pt2 = 2 * (ds.n_src - 3 * ds.n_seg);
    const int n_out = n_pt2 + 4 * ds.n_seg;
    if (n_out > 0) k_agent_reduce<<<n_out, 256, 0, st>>>(slot, val, n, n_pt2, grad_pts, grad_segs);
}

}  // namespace spm
