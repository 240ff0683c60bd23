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

#include <algorithm>

#include <mutex>

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

// The loss, mean agent distance (FP64 sum, fixed order): chunk c of the
// agents is summed by CTA c (each thread its agents a, a + blockDim, ...,
// eight gathers in flight, then a fixed tree), then the chunks in order.
__global__ void __launch_bounds__(256) k_loss_partial(const int32_t *agents, int n, int Nx, int Ny, const float *dist,
                                                      double *partial) {
    __shared__ double part[256];
    const int per = (n + gridDim.x - 1) / gridDim.x, a_lo = blockIdx.x * per, a_hi = min(n, a_lo + per);
    double s = 0.0;
    constexpr int kU = 8;
    for (int a0 = a_lo + threadIdx.x; a0 < a_hi; a0 += kU * blockDim.x) {
        float d[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int a = a0 + u * blockDim.x;
            const int i = a < a_hi ? agents[2 * a] : -1, j = a < a_hi ? agents[2 * a + 1] : -1;
            const bool in = i >= 0 && j >= 0 && i < Nx && j < Ny;
            d[u] = in ? dist[(size_t)j * Nx + i] : INFINITY;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (d[u] < INFINITY) s += (double)d[u];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = part[0];
}

__global__ void k_loss_final(const double *partial, int chunks, int n, float *loss) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += partial[c];
    *loss = (float)(s / (double)max(n, 1));
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

// Gradient of the loss from the agents' contributions, reduced in a fixed
// order so that results are deterministic: agents are cut into `chunks`
// fixed ranges; CTA (o, b) sums component o over range b (a fixed per-thread
// stride, then a fixed tree) into partial[o * chunks + b] (FP64); then one
// thread per component sums its partials in range order.
__global__ void __launch_bounds__(256) k_agent_partial(const int32_t *slot, const float4 *val, int n, int chunks,
                                                       double *partial) {
    __shared__ double part[256];
    const int o = blockIdx.x, b = blockIdx.y;
    const int a0 = (int)((long long)n * b / chunks), a1 = (int)((long long)n * (b + 1) / chunks);
    double s = 0.0;
    for (int a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
        const int sl = slot[a], d = o - sl;
        if (sl < 0 || d < 0 || d > 3) continue;
        const float4 v = val[a];
        s += (double)(d == 0 ? v.x : d == 1 ? v.y : d == 2 ? v.z : v.w);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) part[threadIdx.x] += part[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)o * chunks + b] = part[0];
}

__global__ void k_agent_final(const double *partial, int chunks, int n, int n_out, int n_pt2, float *grad_pts,
                              float *grad_segs) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_out) return;
    double s = 0.0;
    for (int b = 0; b < chunks; ++b) s += partial[(size_t)o * chunks + b];
    const float g = (float)(s / (double)max(n, 1));
    if (o < n_pt2) grad_pts[o] = g;
    else grad_segs[o - n_pt2] = g;
}

}  // namespace

// Agent chunks of the two-level reduction for n_out gradient components:
// at most 64, and at most kGradPartials partial sums in all.
int grad_chunks(int n_out) { return n_out <= 0 ? 1 : max(1, min(64, kGradPartials / n_out)); }

void launch_agents_forward(const DevScene &ds, cudaStream_t st, const int32_t *agents, int n,
                           const float *dist, float *loss, double *partial) {
    const int chunks = std::max(1, std::min(kLossPartials, (n + 2047) / 2048));
    k_loss_partial<<<chunks, 256, 0, st>>>(agents, n, ds.Nx, ds.Ny, dist, partial);
    k_loss_final<<<1, 32, 0, st>>>(partial, chunks, n, loss);
}

void launch_agents_contrib(const DevScene &ds, cudaStream_t st, const int32_t *agents, int n,
                           const int32_t *parent, int32_t *root, float2 *lastpt, int32_t *slot, float4 *val) {
    k_root_table<<<(ds.n_gen + 255) / 256, 256, 0, st>>>(ds, root, lastpt);
    const int blocks = n > 0 ? min((n + 255) / 256, 152 * 8) : 1;
    k_agent_contrib<<<blocks, 256, 0, st>>>(ds, agents, n, parent, root, lastpt, slot, val);
}

void launch_agents_reduce(int n_pts, int n_seg, cudaStream_t st, const int32_t *slot, const float4 *val, int n,
                          double *partial, float *grad_pts, float *grad_segs) {
    const int n_pt2 = 2 * n_pts, n_out = n_pt2 + 4 * n_seg;
    if (n_out <= 0) return;
    const int chunks = grad_chunks(n_out);
    k_agent_partial<<<dim3(n_out, chunks), 256, 0, st>>>(slot, val, n, chunks, partial);
    k_agent_final<<<(n_out + 255) / 256, 256, 0, st>>>(partial, chunks, n, n_out, n_pt2, grad_pts, grad_segs);
}

void launch_agents_backward(const DevScene &ds, cudaStream_t st, const int32_t *agents, int n,
                            const int32_t *parent, int32_t *root, float2 *lastpt, int32_t *slot,
                            float4 *val, double *partial, float *grad_pts, float *grad_segs) {
    launch_agents_contrib(ds, st, agents, n, parent, root, lastpt, slot, val);
    launch_agents_reduce(ds.n_src - 3 * ds.n_seg, ds.n_seg, st, slot, val, n, partial, grad_pts, grad_segs);
}

}  // namespace spm

// ---------------------------------------------------------------------------
// Allocation-free backward (spm_agents_backward_noalloc).
//
// Same kernels and launcher as spm_agents_backward, but the scratch (root
// table, last points, per-agent slots and values) lives in one file-scope
// device array instead of buffers allocated by spm_agents_forward. Every GPU
// that loads the library keeps this array until the process exits. Host code
// must not pass the array's name to a kernel: the host-side symbol is only a
// stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and cached.
// ---------------------------------------------------------------------------
namespace spm {
namespace {

constexpr size_t kNaRootOff = 0;
constexpr size_t kNaLastOff = kNaRootOff + sizeof(int32_t) * SPM_NOALLOC_MAX_GENERATORS;
constexpr size_t kNaSlotOff = kNaLastOff + sizeof(float2) * SPM_NOALLOC_MAX_GENERATORS;
constexpr size_t kNaValOff = kNaSlotOff + sizeof(int32_t) * SPM_NOALLOC_MAX_AGENTS;
constexpr size_t kNaPartOff = kNaValOff + sizeof(float4) * SPM_NOALLOC_MAX_AGENTS;
constexpr size_t kNaBytes = kNaPartOff + sizeof(double) * kGradPartials;
static_assert(kNaLastOff % 16 == 0 && kNaSlotOff % 16 == 0 && kNaValOff % 16 == 0 && kNaPartOff % 16 == 0,
              "alignment");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char *g_na_addr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t noalloc_scratch(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_na_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace spm

extern "C" spm_status spm_agents_backward_noalloc(spm_scene *scene, void *stream,
                                                  const int32_t *agents_dev, int32_t n,
                                                  const int32_t *parent_dev, float *grad_points_dev,
                                                  float *grad_segs_dev) {
    using namespace spm;
    if (!scene) return SPM_ERR_INVALID_ARG;
    const DevScene &ds = *scene_dev(scene);
    const int n_pts = ds.n_src - 3 * ds.n_seg;
    if (n < 0 || (n > 0 && !agents_dev) || !parent_dev || (n_pts > 0 && !grad_points_dev) ||
        (ds.n_seg > 0 && !grad_segs_dev)) {
        scene_set_error(scene, "null pointer or negative agent count");
        return SPM_ERR_INVALID_ARG;
    }
    if (n > SPM_NOALLOC_MAX_AGENTS || ds.n_gen > SPM_NOALLOC_MAX_GENERATORS) {
        scene_set_error(scene, "too many agents or generators for the fixed scratch "
                               "(limits: SPM_NOALLOC_MAX_AGENTS, SPM_NOALLOC_MAX_GENERATORS)");
        return SPM_ERR_CAPACITY;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        scene_set_error(scene, "cudaGetDevice failed");
        return SPM_ERR_CUDA;
    }
    if (dev != scene_device(scene)) {
        scene_set_error(scene, "scene used on another device");
        return SPM_ERR_INVALID_ARG;
    }
    unsigned char *base = nullptr;
    cudaError_t e = noalloc_scratch(dev, &base);
    if (e != cudaSuccess) {
        scene_set_error(scene, cudaGetErrorString(e));
        return SPM_ERR_CUDA;
    }
    // Every scratch element the kernels read is written earlier in the same
    // call (root/lastpt for all generators, slot/val for all n agents, one
    // partial sum per chunk and component), so nothing needs clearing
    // between calls.
    launch_agents_backward(ds, static_cast<cudaStream_t>(stream), agents_dev, n, parent_dev,
                           reinterpret_cast<int32_t *>(base + kNaRootOff),
                           reinterpret_cast<float2 *>(base + kNaLastOff),
                           reinterpret_cast<int32_t *>(base + kNaSlotOff),
                           reinterpret_cast<float4 *>(base + kNaValOff),
                           reinterpret_cast<double *>(base + kNaPartOff), grad_points_dev, grad_segs_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        scene_set_error(scene, cudaGetErrorString(e));
        return SPM_ERR_CUDA;
    }
    return SPM_OK;
}
