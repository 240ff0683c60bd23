// spm_api.cu -- the C ABI (include/spm.h): scene lifetime, device buffers,
// compute entry points and host-side queries.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "spm_internal.h"


struct spm_scene {
    spm::HostScene hs;
    spm::DevScene ds{};
    int device = 0;
    std::string err;
    std::vector<void *> allocs;
    const float *last_dist = nullptr;
    const int32_t *last_parent = nullptr;
    cudaStream_t last_stream = nullptr;
    float *stage_dist = nullptr;  // device staging for spm_compute_host
    int32_t *stage_par = nullptr;
    // differentiable form: root table (built by each forward that records a
    // tape) and the partial sums of the gradient reduction
    int32_t *root = nullptr;
    float2 *lastpt = nullptr;
    double *grad_partial = nullptr;
    double *loss_partial = nullptr;  // the forward loss's chunk sums
    // phase timing events (vertex start, pixel start, end)
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool ev_valid = false;
    double *query_out = nullptr;  // exact query result: distance, then parent (device)
    // side stream of the geometric flood (flood mode 3), with fork/join events
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    spm::VertexSide vside = {nullptr, nullptr, nullptr};  // the edge lists beside the warm start's kernels
    // host-buffer computes: copy stream, one event per pixel-pass slab, and
    // one for the end of the copies
    cudaStream_t copy = nullptr;
    cudaEvent_t slab_ev[8] = {};
    cudaEvent_t copy_done = nullptr;
    // pageable host destinations: two page-locked bounce buffers (dist rows,
    // then parent rows, of the largest slab), filled by the copy stream and
    // emptied by the host while the next slab computes
    unsigned char *bounce[2] = {nullptr, nullptr};
    size_t bounce_bytes = 0;
    cudaEvent_t bounce_ev[2] = {nullptr, nullptr};
    // the device holds sources moved by spm_scene_update_sources_device that
    // the host copy in hs has not seen yet
    bool host_src_stale = false;
    bool alloc_failed = false;  // some device allocation of this scene failed
    int seq_blocks = 0;  // co-resident CTAs of the sequential kernel
    // the static part of the geometric flood (obstacle vertices) is on the
    // device for this tile size and depth-map setting
    bool flood_static_ok = false;
    int flood_static_tile = 0, flood_static_maps = 0;
    // the warm start of the fixpoint: the rounds the table build's deepest
    // root took, whether that makes the warm start the default, and the
    // caller's choice (spm_tuning.fixpoint_start)
    int vtab_depth = 0;
    bool warm_deep = false;
    int fix_start = 0;
};

namespace {

thread_local std::string g_create_err;

spm_status set_err(spm_scene *s, spm_status st, const std::string &msg) {
    if (s) s->err = msg;
    else g_create_err = msg;
    return st;
}

// Test hook (spm_debug_fail_alloc_after): the n-th next device allocation
// fails, so that the failure paths can be exercised; -1 = never.
std::atomic<int> g_fail_alloc_after{-1};

// Host-side NVTX range over a scope: the phases of a compute show up by name
// in a profiler's timeline.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

template <class T>
T *dalloc(spm_scene *s, size_t n) {
    for (int k = g_fail_alloc_after.load(); k >= 0; k = g_fail_alloc_after.load())
        if (g_fail_alloc_after.compare_exchange_weak(k, k - 1)) {
            if (k == 0) {
                s->alloc_failed = true;
                return nullptr;
            }
            break;
        }
    void *p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
        cudaGetLastError();  // not sticky: clear it, the caller reports SPM_ERR_OOM
        s->alloc_failed = true;
        return nullptr;
    }
    s->allocs.push_back(p);
    return static_cast<T *>(p);
}

template <class T>
T *dupload(spm_scene *s, const std::vector<T> &v, bool &ok) {
    T *p = dalloc<T>(s, v.size());
    if (!p) {
        ok = false;
        return nullptr;
    }
    if (!v.empty() && cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        ok = false;
    return p;
}

void free_all(spm_scene *s) {
    for (void *p : s->allocs) cudaFree(p);
    s->allocs.clear();
    for (cudaEvent_t &e : s->ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    for (cudaEvent_t *e : {&s->fork, &s->join, &s->copy_done, &s->vside.fork, &s->vside.join})
        if (*e) {
            cudaEventDestroy(*e);
            *e = nullptr;
        }
    for (cudaEvent_t &e : s->slab_ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    for (int k = 0; k < 2; ++k) {
        if (s->bounce_ev[k]) {
            cudaEventDestroy(s->bounce_ev[k]);
            s->bounce_ev[k] = nullptr;
        }
        if (s->bounce[k]) {
            cudaFreeHost(s->bounce[k]);
            s->bounce[k] = nullptr;
        }
    }
    if (s->copy) {
        cudaStreamDestroy(s->copy);
        s->copy = nullptr;
    }
    if (s->side) {
        cudaStreamDestroy(s->side);
        s->side = nullptr;
    }
    if (s->vside.st) {
        cudaStreamDestroy(s->vside.st);
        s->vside.st = nullptr;
    }
}

spm_status check_device(spm_scene *s) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_err(s, SPM_ERR_CUDA, "cudaGetDevice failed");
    if (dev != s->device) return set_err(s, SPM_ERR_INVALID_ARG, "scene used on another device");
    return SPM_OK;
}

void set_tile(spm::DevScene &ds, int tile) {
    ds.tile = tile;
    ds.tiles_x = (ds.Nx + tile - 1) / tile;
    ds.tiles_y = (ds.Ny + tile - 1) / tile;
}

spm_status upload_sources(spm_scene *s) {
    const spm::HostScene &hs = s->hs;
    spm::DevScene &ds = s->ds;
    std::vector<float> segpos(hs.segs.begin(), hs.segs.end());
    bool ok = true;
    ok &= cudaMemcpy((void *)ds.gen_lat, hs.gen_lat.data(), sizeof(int32_t) * 2 * hs.n_src,
                     cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy((void *)ds.gen_pos, hs.gen_pos.data(), sizeof(float) * 2 * hs.n_src,
                     cudaMemcpyHostToDevice) == cudaSuccess;
    if (!hs.seg_lat.empty()) {
        ok &= cudaMemcpy((void *)ds.seg_lat, hs.seg_lat.data(), sizeof(int32_t) * hs.seg_lat.size(),
                         cudaMemcpyHostToDevice) == cudaSuccess;
        ok &= cudaMemcpy((void *)ds.seg_pos, segpos.data(), sizeof(float) * segpos.size(),
                         cudaMemcpyHostToDevice) == cudaSuccess;
    }
    return ok ? SPM_OK : set_err(s, SPM_ERR_CUDA, "source upload failed");
}

// Brings the host copy of the Source entries up to date after device-side
// updates (synchronises the device).
spm_status refresh_host_sources(spm_scene *s) {
    if (!s->host_src_stale) return SPM_OK;
    spm::HostScene &hs = s->hs;
    const spm::DevScene &ds = s->ds;
    const int np = (int)hs.points.size() / 2, ns = (int)hs.segs.size() / 4;
    if (cudaDeviceSynchronize() != cudaSuccess) return set_err(s, SPM_ERR_CUDA, "synchronisation failed");
    bool ok = true;
    ok &= cudaMemcpy(hs.gen_lat.data(), ds.gen_lat, sizeof(int32_t) * 2 * hs.n_src, cudaMemcpyDeviceToHost) ==
          cudaSuccess;
    ok &= cudaMemcpy(hs.gen_pos.data(), ds.gen_pos, sizeof(float) * 2 * hs.n_src, cudaMemcpyDeviceToHost) ==
          cudaSuccess;
    if (ns) {
        ok &= cudaMemcpy(hs.seg_lat.data(), ds.seg_lat, sizeof(int32_t) * 4 * ns, cudaMemcpyDeviceToHost) ==
              cudaSuccess;
        ok &= cudaMemcpy(hs.segs.data(), ds.seg_pos, sizeof(float) * 4 * ns, cudaMemcpyDeviceToHost) == cudaSuccess;
    }
    if (!ok) return set_err(s, SPM_ERR_CUDA, "source table copy failed");
    for (int i = 0; i < 2 * np; ++i) hs.points[i] = hs.gen_pos[i];
    s->host_src_stale = false;
    return SPM_OK;
}

}  // namespace

extern "C" {

const char *spm_status_string(spm_status st) {
    switch (st) {
    case SPM_OK: return "ok";
    case SPM_ERR_INVALID_ARG: return "invalid argument";
    case SPM_ERR_BAD_GEOMETRY: return "bad geometry";
    case SPM_ERR_OOM: return "out of memory";
    case SPM_ERR_CUDA: return "CUDA error";
    case SPM_ERR_NOT_CONVERGED: return "vertex-cost fixpoint did not converge";
    case SPM_ERR_TIMEOUT: return "device wait timed out";
    case SPM_ERR_CAPACITY: return "device buffer capacity exceeded";
    }
    return "unknown status";
}

const char *spm_last_error(const spm_scene *s) { return s ? s->err.c_str() : g_create_err.c_str(); }

void spm_debug_fail_alloc_after(int32_t n) { g_fail_alloc_after.store(n < 0 ? -1 : n); }

spm_status spm_scene_create(const spm_scene_desc *desc, spm_scene **out) {
    if (!desc || !out) return set_err(nullptr, SPM_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    spm_scene *s = new (std::nothrow) spm_scene();
    if (!s) return set_err(nullptr, SPM_ERR_OOM, "host allocation failed");
    std::string err;
    spm_status st = spm::prepare_scene(*desc, s->hs, err);
    if (st != SPM_OK) {
        delete s;
        return set_err(nullptr, st, err);
    }
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return set_err(nullptr, SPM_ERR_CUDA, "no CUDA device");
    }
    const spm::HostScene &hs = s->hs;
    spm::DevScene &ds = s->ds;
    ds.Wx = hs.Wx; ds.Wy = hs.Wy; ds.Nx = hs.Nx; ds.Ny = hs.Ny; ds.S = hs.S;
    ds.hx = (float)hs.Wx / (float)hs.Nx;
    ds.hy = (float)hs.Wy / (float)hs.Ny;
    ds.n_poly = (int32_t)hs.poly_off.size() - 1;
    ds.n_gen = hs.n_gen; ds.n_src = hs.n_src; ds.n_vert = hs.n_vert;
    ds.n_seg = (int32_t)hs.segs.size() / 4;
    ds.bin_x0 = hs.bin_x0; ds.bin_y0 = hs.bin_y0; ds.bin_size = hs.bin_size;
    ds.bin_nx = hs.bin_nx; ds.bin_ny = hs.bin_ny;
    if (hs.n_gen > (1 << 20)) {
        delete s;
        return set_err(nullptr, SPM_ERR_CAPACITY, "more than 2^20 generators");
    }
    bool ok = true;
    ds.poly_off = dupload(s, hs.poly_off, ok);
    {
        std::vector<int2> v(hs.poly_v.size() / 2);
        std::memcpy(v.data(), hs.poly_v.data(), sizeof(int32_t) * hs.poly_v.size());
        ds.poly_v = dupload(s, v, ok);
        std::vector<int4> b(hs.poly_box.size() / 4);
        std::memcpy(b.data(), hs.poly_box.data(), sizeof(int32_t) * hs.poly_box.size());
        ds.poly_box = dupload(s, b, ok);
    }
    ds.bin_start = dupload(s, hs.bin_start, ok);
    ds.bin_items = dupload(s, hs.bin_items, ok);
    {
        std::vector<spm::BinRec> recs(hs.bin_items.size());
        for (size_t i = 0; i < recs.size(); ++i) {
            const int k = hs.bin_items[i];
            recs[i].box = make_int4(hs.poly_box[4 * k], hs.poly_box[4 * k + 1], hs.poly_box[4 * k + 2],
                                    hs.poly_box[4 * k + 3]);
            recs[i].poly = k;
            recs[i].voff = hs.poly_off[k];
            recs[i].m = hs.poly_off[k + 1] - hs.poly_off[k];
            recs[i].pad = 0;
        }
        ds.bin_recs = dupload(s, recs, ok);
    }
    ds.gen_kind = dupload(s, hs.gen_kind, ok);
    ds.gen_aux = dupload(s, hs.gen_aux, ok);
    {
        std::vector<int2> l(hs.n_gen);
        std::memcpy(l.data(), hs.gen_lat.data(), sizeof(int32_t) * 2 * hs.n_gen);
        ds.gen_lat = dupload(s, l, ok);
        std::vector<float2> p(hs.n_gen);
        std::memcpy(p.data(), hs.gen_pos.data(), sizeof(float) * 2 * hs.n_gen);
        ds.gen_pos = dupload(s, p, ok);
        std::vector<int4> w(hs.n_gen);
        std::memcpy(w.data(), hs.gen_wedge.data(), sizeof(int32_t) * 4 * hs.n_gen);
        ds.gen_wedge = dupload(s, w, ok);
        std::vector<int4> sl(ds.n_seg);
        if (ds.n_seg) std::memcpy(sl.data(), hs.seg_lat.data(), sizeof(int32_t) * 4 * ds.n_seg);
        ds.seg_lat = dupload(s, sl, ok);
        std::vector<float4> sp(ds.n_seg);
        if (ds.n_seg) std::memcpy(sp.data(), hs.segs.data(), sizeof(float) * 4 * ds.n_seg);
        ds.seg_pos = dupload(s, sp, ok);
    }
    ds.vis_words = (hs.n_gen + 31) / 32;
    ds.vis_bits = dalloc<uint32_t>(s, (size_t)hs.n_vert * ds.vis_words);
    // obstacle-vertex pairs are tested once, here; a compute tests the
    // source columns only
    uint32_t *vis_static = dalloc<uint32_t>(s, (size_t)hs.n_vert * ds.vis_words);
    ds.vis_static = vis_static;
    ds.pair_words = (hs.n_src + 31) / 32;
    ds.pair_u0 = 0;
    ds.pair_u1 = hs.n_src;
    ds.in_start = dalloc<int32_t>(s, hs.n_vert + 1);
    ds.out_start = dalloc<int32_t>(s, hs.n_gen + 1);
    ds.out_fill = dalloc<int32_t>(s, hs.n_gen);
    ds.edge_cap = std::min<int64_t>(std::min<int64_t>((int64_t)hs.n_gen * hs.n_vert, (int64_t)1 << 26),
                                    std::max<int64_t>(1 << 20, 128 * (int64_t)hs.n_gen));
    ds.in_src = dalloc<int32_t>(s, ds.edge_cap);
    ds.in_len = dalloc<double>(s, ds.edge_cap);
    ds.out_dst = dalloc<int32_t>(s, ds.edge_cap);
    for (int k = 0; k < 2; ++k) {
        ds.cost[k] = dalloc<double>(s, hs.n_gen);
        ds.par[k] = dalloc<int32_t>(s, hs.n_gen);
        ds.frontier[k] = dalloc<int32_t>(s, hs.n_gen);
        ds.dirtyl[k] = dalloc<int32_t>(s, hs.n_gen);
    }
    ds.gen_costf = dalloc<float>(s, hs.n_gen);
    ds.gen_cost = dalloc<double>(s, hs.n_gen);
    ds.gen_par = dalloc<int32_t>(s, hs.n_gen);
    ds.gen_cone = dalloc<int4>(s, hs.n_gen);
    ds.gen_ctype = dalloc<int32_t>(s, hs.n_gen);
    ds.dirty = dalloc<uint32_t>(s, (hs.n_gen + 31) / 32);
    ds.counters = dalloc<int32_t>(s, 8);
    ds.status = dalloc<uint32_t>(s, 1);
    ds.stats = dalloc<int32_t>(s, 4);
    {
        // lists are sized for the small tile; the default tile follows the pixel size
        const int64_t ntiles = (int64_t)((hs.Nx + spm::kTileSmall - 1) / spm::kTileSmall) *
                               ((hs.Ny + spm::kTileSmall - 1) / spm::kTileSmall);
        set_tile(ds, (ds.hx >= 8.f || ds.hy >= 8.f) ? spm::kTileSmall : spm::kTile);
        ds.use_flood = spm::flood_possible((int)ntiles, ds.n_poly) && spm::flood_smem_attr() ? 1 : 0;
        ds.flood_mode = 0;
        ds.hidden_chunk = 32;
        ds.use_maps = 0;
        const int64_t cap = std::min<int64_t>(std::max<int64_t>((int64_t)hs.n_gen * ntiles, 1),
                                              std::max<int64_t>(4 << 20, 64 * (int64_t)hs.n_gen));
        ds.pair_cap = ds.use_flood ? (int32_t)cap : 1;
        ds.tile_start = dalloc<int32_t>(s, ntiles + 1);
        ds.tile_count = dalloc<int32_t>(s, ntiles);
        ds.tile_items = dalloc<int32_t>(s, ds.pair_cap);
        ds.pairs = dalloc<int2>(s, ds.pair_cap);
        ds.glob_list = dalloc<int32_t>(s, hs.n_gen);
        // depth maps for the pixel pass, when they fit in 256 MB
        const size_t map_bytes = (size_t)hs.n_gen * spm::kAngBins * sizeof(float2);
        ds.gen_maps = nullptr;
        ds.gen_map_ok = nullptr;
        if (ds.use_flood && map_bytes <= ((size_t)256 << 20)) {
            ds.gen_maps = dalloc<float2>(s, (size_t)hs.n_gen * spm::kAngBins);
            ds.gen_map_ok = dalloc<uint8_t>(s, hs.n_gen);
            if (ds.gen_map_ok) cudaMemset(ds.gen_map_ok, 0, hs.n_gen);
        }
        ds.flood_counts = dalloc<int32_t>(s, 4);
        ds.static_tile_start = ds.use_flood ? dalloc<int32_t>(s, ntiles + 1) : nullptr;
        ds.static_tile_items = ds.use_flood ? dalloc<int32_t>(s, ds.pair_cap) : nullptr;
        ds.static_counts = ds.use_flood ? dalloc<int32_t>(s, 4) : nullptr;
        ds.static_lists = 0;
        ds.src_direct = 0;
    }
    ds.free_words = (hs.Nx + 31) / 32;
    uint32_t *free_bits = dalloc<uint32_t>(s, (size_t)hs.Ny * ds.free_words);
    ds.free_bits = free_bits;
    // local depth maps of the obstacle vertices, when they fit in 256 MB
    float *vert_maps = nullptr;
    if ((size_t)hs.n_vert * spm::kLocBins * sizeof(float) <= ((size_t)256 << 20))
        vert_maps = dalloc<float>(s, (size_t)hs.n_vert * spm::kLocBins);
    ds.vert_maps = vert_maps;
    {
        const int n_out = 2 * (hs.n_src - 3 * ds.n_seg) + 4 * ds.n_seg;
        s->root = dalloc<int32_t>(s, hs.n_gen);
        s->lastpt = dalloc<float2>(s, hs.n_gen);
        s->grad_partial = dalloc<double>(s, (size_t)std::max(n_out, 1) * spm::grad_chunks(n_out));
        s->loss_partial = dalloc<double>(s, spm::kLossPartials);
    }
    ds.sssp_blocks = spm::sssp_grid_blocks();
    ds.solo_smem = spm::solo_smem_bytes();
    ok &= !s->alloc_failed;  // no kernel below may run on a buffer that failed to allocate
    if (!ok) {
        free_all(s);
        delete s;
        return set_err(nullptr, SPM_ERR_OOM, "device allocation or upload failed");
    }
    cudaMemset(ds.status, 0, sizeof(uint32_t));
    cudaMemset(ds.stats, 0, sizeof(int32_t) * 4);
    spm::launch_free_mask(ds, nullptr, free_bits);
    if (vert_maps) spm::launch_vert_maps(ds, nullptr, vert_maps);
    spm::launch_vis_static(ds, nullptr, vis_static);  // after the local depth maps it filters with
    // the obstacle-vertex edges are fixed: kept as CSR (in-lists with their
    // lengths, out-lists), so that a compute builds only the sources' edges
    std::vector<int32_t> deg;
    if (ok && hs.n_vert > 0) {
        const int nv = hs.n_vert, ns = hs.n_src, words = ds.vis_words;
        std::vector<uint32_t> bits((size_t)nv * words);
        if (cudaMemcpy(bits.data(), vis_static, sizeof(uint32_t) * bits.size(), cudaMemcpyDeviceToHost) == cudaSuccess) {
            deg.assign(nv, 0);
            std::vector<int32_t> start(nv + 1, 0), out_start(nv + 1, 0), out_init(hs.n_gen + 1, 0);
            for (int vv = 0; vv < nv; ++vv) {
                for (int w = 0; w < words; ++w) {
                    uint32_t b = bits[(size_t)vv * words + w];
                    while (b) {
                        const int u = 32 * w + __builtin_ctz(b);
                        b &= b - 1;
                        if (u < ns) continue;  // no source columns are kept
                        ++deg[vv];
                        ++out_start[u - ns + 1];
                    }
                }
                start[vv + 1] = start[vv] + deg[vv];
            }
            const long long E_s = start[nv];
            if (E_s <= ds.edge_cap) {
                for (int uu = 0; uu < nv; ++uu) {
                    out_init[ns + uu + 1] = out_start[uu + 1];
                    out_start[uu + 1] += out_start[uu];
                }
                std::vector<int32_t> src(E_s > 0 ? E_s : 1), dst(E_s > 0 ? E_s : 1), fill(out_start.begin(), out_start.end() - 1);
                for (int vv = 0; vv < nv; ++vv) {
                    int e = start[vv];
                    for (int w = 0; w < words; ++w) {
                        uint32_t b = bits[(size_t)vv * words + w];
                        while (b) {
                            const int u = 32 * w + __builtin_ctz(b);
                            b &= b - 1;
                            if (u < ns) continue;
                            src[e++] = u;  // increasing generator order, as a compute lists a row
                            dst[fill[u - ns]++] = ns + vv;
                        }
                    }
                }
                ds.st_start = dupload(s, start, ok);
                ds.st_src = dupload(s, src, ok);
                ds.st_out_start = dupload(s, out_start, ok);
                ds.st_out_dst = dupload(s, dst, ok);
                ds.st_out_init = dupload(s, out_init, ok);
                double *len = dalloc<double>(s, E_s > 0 ? E_s : 1);
                ok &= len != nullptr && !s->alloc_failed;
                if (ok) spm::launch_static_lengths(ds, len, nullptr);
                ds.st_len = len;
            }
        }
    }
    if (!ok || s->alloc_failed) {
        free_all(s);
        delete s;
        return set_err(nullptr, SPM_ERR_OOM, "device allocation or upload failed");
    }
    ds.fix_launch = spm::fixpoint_launches(ds, deg);
    // obstacles never move: the geodesic distances between obstacle vertices
    // are tabled once, and every compute starts its fixpoint from the tree
    // they give
    ds.vtab = nullptr;
    ds.warm = 0;
    if (spm::vtab_possible(ds)) {
        const size_t nv = (size_t)hs.n_vert;
        double *tab = dalloc<double>(s, nv * nv);
        int32_t *counter = dalloc<int32_t>(s, 2);  // roots taken, the most rounds a root took
        ds.warm_est = dalloc<double>(s, nv);
        ds.warm_tpar = dalloc<int32_t>(s, nv);
        ds.warm_tlen = dalloc<double>(s, nv);
        ds.warm_cost = dalloc<double>(s, hs.n_gen);
        ds.warm_par = dalloc<int32_t>(s, hs.n_gen);
        int32_t rounds[2] = {0, 0};
        if (!s->alloc_failed && spm::launch_vtab_build(ds, tab, counter, nullptr) == cudaSuccess &&
            cudaMemcpy(rounds, counter, sizeof(rounds), cudaMemcpyDeviceToHost) == cudaSuccess) {
            ds.vtab = tab;
            // a start from the sources takes about as many rounds as the
            // deepest tree has links: the tree pays for itself on deep graphs
            s->vtab_depth = rounds[1];
            s->warm_deep = rounds[1] >= spm::kWarmMinDepth;
            ds.warm = s->warm_deep ? 1 : 0;
        }
    }
    if (s->alloc_failed) {
        free_all(s);
        delete s;
        return set_err(nullptr, SPM_ERR_OOM, "device allocation or upload failed");
    }
    if (cudaPeekAtLastError() != cudaSuccess) {
        free_all(s);
        delete s;
        return set_err(nullptr, SPM_ERR_CUDA, "scene preparation kernels failed to launch");
    }
    for (cudaEvent_t &e : s->ev)
        if (cudaEventCreate(&e) != cudaSuccess) ok = false;
    if (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->copy_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->vside.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->vside.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->vside.join, cudaEventDisableTiming) != cudaSuccess)
        ok = false;
    for (cudaEvent_t &e : s->slab_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) ok = false;
    if (!ok) {
        free_all(s);
        delete s;
        return set_err(nullptr, SPM_ERR_CUDA, "event creation failed");
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_all(s);
        delete s;
        return set_err(nullptr, SPM_ERR_CUDA, "device synchronisation failed");
    }
    *out = s;
    return SPM_OK;
}

void spm_scene_destroy(spm_scene *s) {
    if (!s) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    free_all(s);
    if (cur >= 0 && cur != s->device) cudaSetDevice(cur);
    delete s;
}

spm_status spm_scene_update_sources(spm_scene *s, const float *pts, const float *segs) {
    if (!s) return set_err(nullptr, SPM_ERR_INVALID_ARG, "null scene");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    std::string err;
    st = spm::update_sources(s->hs, pts, segs, err);
    if (st != SPM_OK) return set_err(s, st, err);
    if (cudaDeviceSynchronize() != cudaSuccess) return set_err(s, SPM_ERR_CUDA, "synchronisation failed");
    s->host_src_stale = false;
    return upload_sources(s);
}

spm_status spm_scene_update_sources_device(spm_scene *s, void *stream, const float *pts_dev,
                                           const float *segs_dev) {
    if (!s) return set_err(nullptr, SPM_ERR_INVALID_ARG, "null scene");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    const int np = (int)s->hs.points.size() / 2, ns = (int)s->hs.segs.size() / 4;
    if ((np > 0 && !pts_dev) || (ns > 0 && !segs_dev)) return set_err(s, SPM_ERR_INVALID_ARG, "null source array");
    spm::launch_update_sources(s->ds, static_cast<cudaStream_t>(stream), pts_dev, segs_dev);
    if (cudaPeekAtLastError() != cudaSuccess) return set_err(s, SPM_ERR_CUDA, "source update launch failed");
    s->host_src_stale = true;
    return SPM_OK;
}

// dist / parent: device planes; when dist_host / parent_host are given (a
// host-buffer compute of the whole grid into pageable memory), the pixel pass
// runs as row slabs: each slab's rows go to a page-locked bounce buffer on the
// copy stream while the next slab computes, and the host moves the previous
// slab from its bounce buffer into the caller's memory meanwhile. Returns
// once every row is in place.
static spm_status compute_impl(spm_scene *s, void *stream, float *dist, int32_t *parent, int tile_row0, int tile_row1,
                        float *dist_host = nullptr, int32_t *parent_host = nullptr) {
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(cs, &cap);
    const bool timed = cap == cudaStreamCaptureStatusNone;
    const bool side = s->ds.use_flood && s->ds.flood_mode == 3;  // geometric flood beside the vertex phase
    s->ds.static_lists = side && s->ds.static_tile_start ? 1 : 0;  // the pixel pass reads the kept lists too
    NvtxRange range_all("spm_compute");
    if (timed) cudaEventRecord(s->ev[0], cs);
    // the geometric flood needs nothing from the vertex phase (costs and
    // cones are applied by the pixel pass): it forks at the start and runs
    // beside the whole vertex chain
    if (side) cudaEventRecord(s->fork, cs);
    {
        NvtxRange r("spm vertex phase");
        spm::launch_vertex_phase(s->ds, cs, &s->vside);
    }
    if (side) {
        NvtxRange r("spm flood (side stream)");
        // the obstacle vertices' flood depends on the obstacles alone: built
        // once for this tile size and map setting, then only the sources flood
        const bool maps = s->ds.use_maps && s->ds.gen_maps;
        const bool reuse = s->flood_static_ok && s->flood_static_tile == s->ds.tile &&
                           s->flood_static_maps == (int)maps && s->ds.static_tile_start;
        cudaStreamWaitEvent(s->side, s->fork, 0);
        spm::launch_flood(s->ds, s->side,
                          !s->ds.static_tile_start ? spm::FloodStatic::kNone
                          : reuse                  ? spm::FloodStatic::kReuse
                                                   : spm::FloodStatic::kBuild);
        cudaEventRecord(s->join, s->side);
        s->flood_static_ok = s->ds.static_tile_start != nullptr;
        s->flood_static_tile = s->ds.tile;
        s->flood_static_maps = (int)maps;
    }
    if (timed) cudaEventRecord(s->ev[1], cs);
    if (side) {
        cudaStreamWaitEvent(cs, s->join, 0);
    } else if (s->ds.use_flood) {
        spm::launch_flood(s->ds, cs);
        s->flood_static_ok = false;  // the lists and maps now hold this flood's
    } else {
        static const int32_t off[4] = {0, 0, 1, 0};
        cudaMemcpyAsync(s->ds.flood_counts, off, sizeof off, cudaMemcpyHostToDevice, cs);
    }
    if (timed) cudaEventRecord(s->ev[3], cs);
    if (!dist_host) {
        NvtxRange r("spm pixel phase");
        spm::launch_pixel_phase(s->ds, cs, dist, parent, tile_row0, tile_row1);
    } else {
        NvtxRange r("spm pixel phase with host copies");
        const int rows = tile_row1 - tile_row0, nslab = std::min(rows, (int)(sizeof s->slab_ev / sizeof s->slab_ev[0]));
        const size_t Nx = (size_t)s->hs.Nx, Ny = (size_t)s->hs.Ny;
        auto slab_rows = [&](int k, size_t &r0, size_t &r1) {
            const int t0 = tile_row0 + rows * k / nslab, t1 = tile_row0 + rows * (k + 1) / nslab;
            r0 = (size_t)t0 * s->ds.tile;
            r1 = std::min((size_t)t1 * s->ds.tile, Ny);
        };
        auto drain = [&](int k) {  // host: slab k from its bounce buffer into the caller's planes
            size_t r0, r1;
            slab_rows(k, r0, r1);
            const size_t cnt = (r1 - r0) * Nx;
            cudaEventSynchronize(s->bounce_ev[k & 1]);
            std::memcpy(dist_host + r0 * Nx, s->bounce[k & 1], sizeof(float) * cnt);
            std::memcpy(parent_host + r0 * Nx, s->bounce[k & 1] + sizeof(float) * cnt, sizeof(int32_t) * cnt);
        };
        for (int k = 0; k < nslab; ++k) {
            const int t0 = tile_row0 + rows * k / nslab, t1 = tile_row0 + rows * (k + 1) / nslab;
            spm::launch_pixel_phase(s->ds, cs, dist, parent, t0, t1);
            cudaEventRecord(s->slab_ev[k], cs);
            cudaStreamWaitEvent(s->copy, s->slab_ev[k], 0);
            size_t r0, r1;
            slab_rows(k, r0, r1);
            const size_t off = r0 * Nx, cnt = (r1 - r0) * Nx;
            // bounce buffer k & 1 was emptied by the host when slab k - 2 drained
            cudaMemcpyAsync(s->bounce[k & 1], dist + off, sizeof(float) * cnt, cudaMemcpyDeviceToHost, s->copy);
            cudaMemcpyAsync(s->bounce[k & 1] + sizeof(float) * cnt, parent + off, sizeof(int32_t) * cnt,
                            cudaMemcpyDeviceToHost, s->copy);
            cudaEventRecord(s->bounce_ev[k & 1], s->copy);
            if (k > 0) drain(k - 1);
        }
        if (nslab > 0) drain(nslab - 1);
    }
    if (timed) cudaEventRecord(s->ev[2], cs);
    s->ev_valid = timed;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(s, SPM_ERR_CUDA, cudaGetErrorString(e));
    const bool whole = tile_row0 == 0 && tile_row1 == s->ds.tiles_y;
    s->last_dist = whole ? dist : nullptr;  // queries need the whole field
    s->last_parent = whole ? parent : nullptr;
    s->last_stream = cs;
    return SPM_OK;
}

spm_status spm_compute(spm_scene *s, void *stream, float *dist, int32_t *parent) {
    if (!s || !dist || !parent) return set_err(s, SPM_ERR_INVALID_ARG, "null argument");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    return compute_impl(s, stream, dist, parent, 0, s->ds.tiles_y);
}

spm_status spm_compute_rows(spm_scene *s, void *stream, int32_t row0, int32_t row1, float *dist, int32_t *parent) {
    if (!s || !dist || !parent) return set_err(s, SPM_ERR_INVALID_ARG, "null argument");
    const int T = s->ds.tile, Ny = s->ds.Ny;
    if (row0 < 0 || row1 > Ny || row0 > row1 || row0 % T != 0 || (row1 % T != 0 && row1 != Ny))
        return set_err(s, SPM_ERR_INVALID_ARG, "rows must be tile-aligned within the grid");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    return compute_impl(s, stream, dist, parent, row0 / T, (row1 + T - 1) / T);
}

spm_status spm_scene_sync(spm_scene *s, void *stream) {
    if (!s) return set_err(nullptr, SPM_ERR_INVALID_ARG, "null scene");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return set_err(s, SPM_ERR_CUDA, cudaGetErrorString(e));
    uint32_t bits = 0;
    if (cudaMemcpy(&bits, s->ds.status, sizeof bits, cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_err(s, SPM_ERR_CUDA, "status read failed");
    if (bits) cudaMemset(s->ds.status, 0, sizeof bits);
    if (bits & spm::kStEdgeOverflow) return set_err(s, SPM_ERR_CAPACITY, "visibility graph exceeds edge capacity");
    if (bits & spm::kStNotConverged) return set_err(s, SPM_ERR_NOT_CONVERGED, "vertex fixpoint hit its round cap");
    if (bits & spm::kStTimeout) return set_err(s, SPM_ERR_TIMEOUT, "device wait gave up");
    if (bits & spm::kStBadSource)
        return set_err(s, SPM_ERR_BAD_GEOMETRY, "device source update rejected: a source is outside the world, "
                                                "not strictly outside every obstacle, or a zero-length segment");
    if (bits) return set_err(s, SPM_ERR_CUDA, "device reported bad input");
    return SPM_OK;
}

spm_status spm_compute_sequential(spm_scene *s, void *stream, float *dist, int32_t *parent) {
    if (!s || !dist || !parent) return set_err(s, SPM_ERR_INVALID_ARG, "null argument");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    if (s->hs.n_gen > spm::kSeqMaxGen) return set_err(s, SPM_ERR_CAPACITY, "more generators than the sequential kernel takes");
    if (!s->seq_blocks) s->seq_blocks = spm::sequential_grid_blocks();
    if (spm::launch_sequential(s->ds, static_cast<cudaStream_t>(stream), dist, parent, s->seq_blocks) != cudaSuccess)
        return set_err(s, SPM_ERR_CUDA, "sequential kernel launch failed");
    return SPM_OK;
}

// Device staging planes for host-buffer computes and the autotuner
// (allocated on first use).
static spm_status ensure_stage(spm_scene *s) {
    if (s->stage_dist) return SPM_OK;
    const size_t npx = (size_t)s->hs.Nx * s->hs.Ny;
    s->stage_dist = dalloc<float>(s, npx);
    s->stage_par = dalloc<int32_t>(s, npx);
    if (!s->stage_dist || !s->stage_par) {
        s->stage_dist = nullptr;
        s->stage_par = nullptr;
        return set_err(s, SPM_ERR_OOM, "staging allocation failed");
    }
    return SPM_OK;
}

spm_status spm_compute_host(spm_scene *s, void *stream, float *dist_host, int32_t *parent_host) {
    if (!s || !dist_host || !parent_host) return set_err(s, SPM_ERR_INVALID_ARG, "null argument");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    // page-locked host buffers are device-addressable: the pixel pass then
    // writes the map straight into them (no staging planes, no copies)
    cudaPointerAttributes ad{}, ap{};
    const bool direct = cudaPointerGetAttributes(&ad, dist_host) == cudaSuccess &&
                        cudaPointerGetAttributes(&ap, parent_host) == cudaSuccess && ad.type == cudaMemoryTypeHost &&
                        ap.type == cudaMemoryTypeHost && ad.devicePointer && ap.devicePointer;
    cudaGetLastError();  // a pageable pointer is not an error here
    if (direct) {
        st = compute_impl(s, stream, static_cast<float *>(ad.devicePointer), static_cast<int32_t *>(ap.devicePointer),
                          0, s->ds.tiles_y);
        // the caller may unpin or free these buffers at any time after the
        // call: queries must not read them (they need a device compute)
        s->last_dist = nullptr;
        s->last_parent = nullptr;
    } else {
        st = ensure_stage(s);
        if (st != SPM_OK) return st;
        const size_t slab_rows = (size_t)((s->ds.tiles_y + 7) / 8 + 1) * s->ds.tile;
        const size_t need = slab_rows * (size_t)s->hs.Nx * (sizeof(float) + sizeof(int32_t));
        if (s->bounce_bytes < need) {  // page-locked bounce buffers, on first use or growth
            for (int k = 0; k < 2; ++k)
                if (s->bounce[k]) {
                    cudaFreeHost(s->bounce[k]);
                    s->bounce[k] = nullptr;
                }
            s->bounce_bytes = 0;
            for (int k = 0; k < 2; ++k) {
                if (cudaHostAlloc((void **)&s->bounce[k], need, cudaHostAllocDefault) != cudaSuccess) {
                    cudaGetLastError();
                    return set_err(s, SPM_ERR_OOM, "page-locked bounce buffer allocation failed");
                }
                if (!s->bounce_ev[k] && cudaEventCreateWithFlags(&s->bounce_ev[k], cudaEventDisableTiming) != cudaSuccess)
                    return set_err(s, SPM_ERR_CUDA, "event creation failed");
            }
            s->bounce_bytes = need;
        }
        st = compute_impl(s, stream, s->stage_dist, s->stage_par, 0, s->ds.tiles_y, dist_host, parent_host);
    }
    if (st != SPM_OK) return st;
    return spm_scene_sync(s, stream);
}

}  // extern "C"

struct spm_batch {
    std::vector<spm_scene *> scenes;
    std::vector<spm::DevScene> descs;  // the scenes' descriptors as the batch runs them
    int device = 0;
    std::vector<void *> allocs;
    spm::BatchDev dev{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;  // the graph runs here, ordered with the caller's stream by events
    cudaEvent_t fork = nullptr, join = nullptr;
    bool capture_failed = false;
    // phase events (start, vertex phase and flood done, end), recorded as
    // event nodes of the batch's graph
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    bool ev_valid = false;
    long long src_ins = 0, src_tiles = 0;  // warp tasks of the sources' direct culling
};

namespace {
template <class T>
T *balloc(spm_batch *b, size_t n) {
    void *p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * (n ? n : 1)) != cudaSuccess) return nullptr;
    b->allocs.push_back(p);
    return static_cast<T *>(p);
}
template <class T>
T *bupload(spm_batch *b, const std::vector<T> &v, bool &ok) {
    T *p = balloc<T>(b, v.size());
    if (!p) {
        ok = false;
        return nullptr;
    }
    if (!v.empty() && cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
    return p;
}
void batch_free(spm_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t *e : {&b->ev[0], &b->ev[1], &b->ev[2], &b->fork, &b->join})
        if (*e) {
            cudaEventDestroy(*e);
            *e = nullptr;
        }
    if (b->graph_stream) {
        cudaStreamDestroy(b->graph_stream);
        b->graph_stream = nullptr;
    }
    for (void *p : b->allocs) cudaFree(p);
    b->allocs.clear();
}
// Builds the static part of the geometric flood (obstacle vertices) that
// descriptor d -- the scene's own or a batch's copy -- reads, and waits.
bool build_flood_static(spm_scene *s, const spm::DevScene &d) {
    spm::launch_flood(d, nullptr, spm::FloodStatic::kBuild);
    if (cudaStreamSynchronize(nullptr) != cudaSuccess) return false;
    s->flood_static_ok = true;
    s->flood_static_tile = d.tile;
    s->flood_static_maps = d.use_maps && d.gen_maps ? 1 : 0;
    return true;
}

bool flood_static_matches(const spm_scene *s, const spm::DevScene &d) {
    return s->flood_static_ok && s->flood_static_tile == d.tile &&
           s->flood_static_maps == (d.use_maps && d.gen_maps ? 1 : 0);
}

void batch_launch(spm_batch *b, cudaStream_t st, bool capturing) {
    // while capturing, external records become event nodes of the graph
    auto rec = [&](cudaEvent_t e) {
        if (capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
        else cudaEventRecord(e, st);
    };
    rec(b->ev[0]);
    spm::launch_vertex_phase_batched(b->dev, st);
    spm::launch_flood_batched(b->dev, st, b->src_ins, b->src_tiles);
    rec(b->ev[1]);
    spm::launch_pixel_phase_batched(b->dev, st);
    rec(b->ev[2]);
}
}  // namespace

extern "C" {

spm_status spm_batch_create(spm_scene *const *scenes, int32_t n, float *const *dist, int32_t *const *parent,
                            spm_batch **out) {
    if (!out || n <= 0 || !scenes || !dist || !parent) return set_err(nullptr, SPM_ERR_INVALID_ARG, "bad argument");
    *out = nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_err(nullptr, SPM_ERR_CUDA, "no CUDA device");
    for (int k = 0; k < n; ++k)
        if (!scenes[k] || !dist[k] || !parent[k] || scenes[k]->device != dev)
            return set_err(nullptr, SPM_ERR_INVALID_ARG, "null scene/buffer or scene on another device");
    spm_batch *b = new (std::nothrow) spm_batch();
    if (!b) return set_err(nullptr, SPM_ERR_OOM, "host allocation failed");
    b->scenes.assign(scenes, scenes + n);
    b->device = dev;
    std::vector<spm::DevScene> descs(n);
    std::vector<long long> pair_off(n + 1, 0), src_map_off(n + 1, 0), src_ins_off(n + 1, 0),
        src_tile_off(n + 1, 0);
    std::vector<int32_t> vert_off(n + 1, 0), gen_off(n + 1, 0), order(n), tile_off(n + 1, 0), flood_off(n + 1, 0);
    std::vector<float *> dv(dist, dist + n);
    std::vector<int32_t *> pv(parent, parent + n);
    int max_gen = 0;
    for (int k = 0; k < n; ++k) {
        descs[k] = scenes[k]->ds;
        descs[k].warm = 0;  // the batched fixpoint starts every scene from its sources
        // geometric floods reuse the obstacle vertices' static lists: built
        // here if the scene has none for this tile size and map setting
        descs[k].flood_reuse = 0;
        if (descs[k].use_flood && descs[k].flood_mode == 3 && descs[k].static_tile_start) {
            if (!flood_static_matches(scenes[k], descs[k]) && !build_flood_static(scenes[k], descs[k])) {
                delete b;
                return set_err(nullptr, SPM_ERR_CUDA, "static flood build failed");
            }
            descs[k].flood_reuse = 1;
        }
        descs[k].static_lists = descs[k].flood_reuse;
        // reusing scenes cull their sources directly where the maps allow it
        const spm::DevScene &d = descs[k];
        descs[k].src_direct = d.flood_reuse && spm::flood_sources_direct(d) ? 1 : 0;
        const long long direct = descs[k].src_direct, ntl = (long long)d.tiles_x * d.tiles_y;
        src_map_off[k + 1] = src_map_off[k] + direct * d.n_src * spm::kAngBins;
        src_ins_off[k + 1] = src_ins_off[k] + direct * d.n_src * d.n_poly;
        src_tile_off[k + 1] = src_tile_off[k] + direct * d.n_src * ntl;
        const bool floods = d.use_flood && d.flood_mode != 2;
        flood_off[k + 1] =
            flood_off[k] + (floods && !direct ? (d.flood_reuse ? d.n_src : d.n_gen) : 0);
        pair_off[k + 1] = pair_off[k] + (long long)descs[k].n_vert * descs[k].pair_words;
        vert_off[k + 1] = vert_off[k] + descs[k].n_vert;
        gen_off[k + 1] = gen_off[k] + descs[k].n_gen;
        max_gen = std::max(max_gen, descs[k].n_gen);
        order[k] = k;
    }
    // the pixel pass takes tiles in this order: the costliest tiles first, so
    // that the kernel's tail is short. A tile's candidates grow with the
    // generators and with the share of the scene the tile covers: estimate
    // its cost by n_gen / sqrt(tiles)
    auto tile_cost = [&](int k) {
        return (double)descs[k].n_gen / std::sqrt((double)std::max(1, descs[k].tiles_x * descs[k].tiles_y));
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return tile_cost(a) > tile_cost(c); });
    for (int k = 0; k < n; ++k)
        tile_off[k + 1] = tile_off[k] + descs[order[k]].tiles_x * descs[order[k]].tiles_y;
    bool ok = true;
    spm::BatchDev &bd = b->dev;
    bd.n = n;
    bd.scenes = bupload(b, descs, ok);
    bd.pair_off = bupload(b, pair_off, ok);
    bd.vert_off = bupload(b, vert_off, ok);
    bd.gen_off = bupload(b, gen_off, ok);
    bd.flood_off = bupload(b, flood_off, ok);
    bd.walk_tasks = flood_off[n];
    bd.src_map_off = bupload(b, src_map_off, ok);
    bd.src_ins_off = bupload(b, src_ins_off, ok);
    bd.src_tile_off = bupload(b, src_tile_off, ok);
    b->src_ins = src_ins_off[n];
    b->src_tiles = src_tile_off[n];
    bd.order = bupload(b, order, ok);
    bd.tile_off = bupload(b, tile_off, ok);
    bd.total_tiles = tile_off[n];
    bd.tile_counter = balloc<int32_t>(b, 1);
    bd.dist = bupload(b, dv, ok);
    bd.parent = bupload(b, pv, ok);
    for (int k = 0; k < 2; ++k) {
        bd.dirtyl[k] = balloc<int2>(b, gen_off[n]);
        bd.frontier[k] = balloc<int2>(b, gen_off[n]);
    }
    bd.counters = balloc<int32_t>(b, 8);
    {  // the vertex fixpoint on resident clusters, most generators first
        std::vector<int32_t> cl_order(n);
        for (int k = 0; k < n; ++k) cl_order[k] = k;
        std::stable_sort(cl_order.begin(), cl_order.end(),
                         [&](int a, int c) { return descs[a].n_gen > descs[c].n_gen; });
        bd.cl_order = bupload(b, cl_order, ok);
        bd.cl_done = balloc<int32_t>(b, n);
        bd.cl_counter = balloc<int32_t>(b, 1);
        bd.cl_grid = spm::cluster_batched_grid();
        bd.cl_all = bd.cl_grid > 0 ? 1 : 0;
        for (int k = 0; k < n; ++k) bd.cl_all &= (descs[k].fix_launch & spm::kFixClusterFits) ? 1 : 0;
    }
    bd.max_rounds = spm::fixpoint_round_cap(max_gen);
    bd.sssp_blocks = spm::sssp_batched_grid_blocks();
    bd.flood_smem = 0;
    bd.any_maps = 0;
    for (int k = 0; k < n; ++k) bd.any_maps |= descs[k].use_flood && descs[k].flood_mode != 2 && descs[k].use_maps;
    for (int k = 0; k < n; ++k)
        if (descs[k].use_flood && descs[k].flood_mode != 2)
            bd.flood_smem = std::max<int32_t>(
                bd.flood_smem, (int32_t)spm::flood_smem_bytes(descs[k].tiles_x * descs[k].tiles_y, descs[k].n_poly,
                                                              descs[k].use_maps && descs[k].gen_maps));
    for (void *p : b->allocs) ok &= p != nullptr;
    if (!ok) {
        batch_free(b);
        delete b;
        return set_err(nullptr, SPM_ERR_OOM, "batch allocation failed");
    }
    for (cudaEvent_t &e : b->ev)
        if (cudaEventCreate(&e) != cudaSuccess) ok = false;
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->graph_stream, cudaStreamNonBlocking) != cudaSuccess)
        ok = false;
    if (!ok) {
        batch_free(b);
        delete b;
        return set_err(nullptr, SPM_ERR_CUDA, "event creation failed");
    }
    b->descs = descs;
    *out = b;
    return SPM_OK;
}

spm_status spm_batch_compute(spm_batch *b, void *stream) {
    if (!b) return set_err(nullptr, SPM_ERR_INVALID_ARG, "null batch");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
        return set_err(nullptr, SPM_ERR_INVALID_ARG, "batch used on another device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // a single-scene compute in another flood mode may have replaced a
    // scene's static lists since: rebuild them before the batch reads them
    for (size_t k = 0; k < b->scenes.size(); ++k)
        if (b->descs[k].flood_reuse && !flood_static_matches(b->scenes[k], b->descs[k])) {
            if (cudaStreamSynchronize(st) != cudaSuccess || !build_flood_static(b->scenes[k], b->descs[k]))
                return set_err(nullptr, SPM_ERR_CUDA, "static flood rebuild failed");
        }
    // the caller's stream may be the legacy default stream, which cannot be
    // captured: the graph is captured and replayed on the batch's own
    // stream, after the caller's prior work and before its later work
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    if (cap != cudaStreamCaptureStatusNone) {  // inside the caller's own capture: record the launches there
        batch_launch(b, st, true);
    } else {
        cudaEventRecord(b->fork, st);
        cudaStreamWaitEvent(b->graph_stream, b->fork, 0);
        if (!b->exec && !b->capture_failed) {  // capture once into a CUDA graph
            cudaGraph_t g = nullptr;
            bool okc = cudaStreamBeginCapture(b->graph_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (okc) {
                batch_launch(b, b->graph_stream, true);
                okc = cudaStreamEndCapture(b->graph_stream, &g) == cudaSuccess && g != nullptr;
            }
            if (okc && cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess) {
                b->graph = g;
            } else {
                if (g) cudaGraphDestroy(g);
                b->exec = nullptr;
                b->capture_failed = true;
                cudaGetLastError();  // clear a capture error; fall back to direct launches
            }
        }
        if (b->exec) {
            if (cudaGraphLaunch(b->exec, b->graph_stream) != cudaSuccess)
                return set_err(nullptr, SPM_ERR_CUDA, "graph launch failed");
        } else {
            batch_launch(b, b->graph_stream, false);
        }
        cudaEventRecord(b->join, b->graph_stream);
        cudaStreamWaitEvent(st, b->join, 0);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(nullptr, SPM_ERR_CUDA, cudaGetErrorString(e));
    b->ev_valid = true;
    for (size_t k = 0; k < b->scenes.size(); ++k) {
        spm_scene *s = b->scenes[k];
        s->last_dist = nullptr;  // queries need a single-scene compute
        s->last_parent = nullptr;
        s->ev_valid = false;
        // the batched flood rewrote the lists of scenes that flood every generator
        if (!b->descs[k].flood_reuse && b->descs[k].use_flood && b->descs[k].flood_mode != 2)
            s->flood_static_ok = false;
    }
    return SPM_OK;
}

spm_status spm_batch_phase_ms(spm_batch *b, float *vertex_ms, float *pixel_ms) {
    if (!b || !vertex_ms || !pixel_ms) return set_err(nullptr, SPM_ERR_INVALID_ARG, "null argument");
    if (!b->ev_valid) return set_err(nullptr, SPM_ERR_INVALID_ARG, "no batch compute recorded");
    if (cudaEventSynchronize(b->ev[2]) != cudaSuccess || cudaEventElapsedTime(vertex_ms, b->ev[0], b->ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(pixel_ms, b->ev[1], b->ev[2]) != cudaSuccess)
        return set_err(nullptr, SPM_ERR_CUDA, "event timing failed");
    return SPM_OK;
}

void spm_batch_destroy(spm_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    batch_free(b);
    delete b;
}

spm_status spm_compute_batched(spm_scene *const *scenes, int32_t n, void *stream, float *const *dist,
                               int32_t *const *parent) {
    if (n == 0) return SPM_OK;
    spm_batch *b = nullptr;
    spm_status st = spm_batch_create(scenes, n, dist, parent, &b);
    if (st != SPM_OK) return st;
    st = spm_batch_compute(b, stream);
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess && st == SPM_OK)
        st = set_err(nullptr, SPM_ERR_CUDA, "synchronisation failed");
    spm_batch_destroy(b);
    return st;
}

spm_status spm_query_parent(spm_scene *s, float x, float y, int32_t *parent, float *dist) {
    if (!s || !parent || !dist) return set_err(s, SPM_ERR_INVALID_ARG, "null argument");
    if (!s->last_dist) return set_err(s, SPM_ERR_INVALID_ARG, "nothing computed yet");
    if (!(x >= 0.f && y >= 0.f && x < (float)s->hs.Wx && y < (float)s->hs.Wy))
        return set_err(s, SPM_ERR_INVALID_ARG, "query point outside the world");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    int i = (int)std::floor(x / s->ds.hx), j = (int)std::floor(y / s->ds.hy);
    i = std::min(i, s->hs.Nx - 1);
    j = std::min(j, s->hs.Ny - 1);
    const size_t idx = (size_t)j * s->hs.Nx + i;
    if (cudaStreamSynchronize(s->last_stream) != cudaSuccess ||
        cudaMemcpy(parent, s->last_parent + idx, sizeof(int32_t), cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(dist, s->last_dist + idx, sizeof(float), cudaMemcpyDefault) != cudaSuccess)
        return set_err(s, SPM_ERR_CUDA, "query copy failed");
    return SPM_OK;
}

spm_status spm_query_exact(spm_scene *s, float x, float y, int32_t *parent, float *dist) {
    if (!s || !parent || !dist) return set_err(s, SPM_ERR_INVALID_ARG, "null argument");
    if (!s->last_parent) return set_err(s, SPM_ERR_INVALID_ARG, "nothing computed yet");
    if (!(x >= 0.f && y >= 0.f && x < (float)s->hs.Wx && y < (float)s->hs.Wy))
        return set_err(s, SPM_ERR_INVALID_ARG, "query point outside the world");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    int i = (int)std::floor(x / s->ds.hx), j = (int)std::floor(y / s->ds.hy);
    i = std::min(i, s->hs.Nx - 1);
    j = std::min(j, s->hs.Ny - 1);
    // the predicates run on the lattice point nearest to (x, y)
    const double S = (double)s->hs.S;
    const int qx = (int)std::lrint((double)x * S), qy = (int)std::lrint((double)y * S);
    if (!s->query_out) {
        s->query_out = dalloc<double>(s, 2);
        if (!s->query_out) return set_err(s, SPM_ERR_OOM, "query buffer allocation failed");
    }
    int32_t *out_par = reinterpret_cast<int32_t *>(s->query_out + 1);
    spm::launch_query_exact(s->ds, s->last_stream, s->last_parent, i, j, qx, qy, (double)x, (double)y, out_par,
                            s->query_out);
    double res[2];
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s->last_stream) != cudaSuccess ||
        cudaMemcpy(res, s->query_out, sizeof res, cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_err(s, SPM_ERR_CUDA, "exact query failed");
    std::memcpy(parent, &res[1], sizeof(int32_t));
    *dist = (float)res[0];
    return SPM_OK;
}

spm_status spm_extract_path(spm_scene *s, float x, float y, float *out_xy, int32_t cap, int32_t *n) {
    if (!s || !out_xy || !n || cap < 1) return set_err(s, SPM_ERR_INVALID_ARG, "bad argument");
    int32_t g;
    float d;
    spm_status st = spm_query_parent(s, x, y, &g, &d);
    if (st != SPM_OK) return st;
    st = refresh_host_sources(s);
    if (st != SPM_OK) return st;
    std::vector<int32_t> par(s->hs.n_gen);
    if (cudaMemcpy(par.data(), s->ds.gen_par, sizeof(int32_t) * s->hs.n_gen, cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_err(s, SPM_ERR_CUDA, "parent table copy failed");
    int cnt = 0;
    out_xy[0] = x;
    out_xy[1] = y;
    cnt = 1;
    float lx = x, ly = y;
    const spm::HostScene &hs = s->hs;
    for (int guard = 0; g >= 0 && guard <= hs.n_gen + 1; ++guard) {
        if (cnt >= cap) return set_err(s, SPM_ERR_CAPACITY, "path longer than cap");
        const int kind = hs.gen_kind[g];
        if (kind == spm::kSegI) {
            const float *F = &hs.segs[4 * hs.gen_aux[g]];
            const float ux = F[2] - F[0], uy = F[3] - F[1];
            const float t = ((lx - F[0]) * ux + (ly - F[1]) * uy) / (ux * ux + uy * uy);
            out_xy[2 * cnt] = F[0] + t * ux;
            out_xy[2 * cnt + 1] = F[1] + t * uy;
            ++cnt;
            break;
        }
        lx = hs.gen_pos[2 * g];
        ly = hs.gen_pos[2 * g + 1];
        out_xy[2 * cnt] = lx;
        out_xy[2 * cnt + 1] = ly;
        ++cnt;
        if (kind != spm::kVert) break;
        g = par[g];
    }
    *n = cnt;
    return SPM_OK;
}

spm_status spm_scene_generators(spm_scene *s, int32_t *kind, int32_t *lattice_xy, double *cost, int32_t *parent) {
    if (!s) return set_err(nullptr, SPM_ERR_INVALID_ARG, "null scene");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    st = refresh_host_sources(s);
    if (st != SPM_OK) return st;
    const int n = s->hs.n_gen;
    if (kind) std::memcpy(kind, s->hs.gen_kind.data(), sizeof(int32_t) * n);
    if (lattice_xy) std::memcpy(lattice_xy, s->hs.gen_lat.data(), sizeof(int32_t) * 2 * n);
    if (cudaDeviceSynchronize() != cudaSuccess) return set_err(s, SPM_ERR_CUDA, "synchronisation failed");
    if (cost && cudaMemcpy(cost, s->ds.gen_cost, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_err(s, SPM_ERR_CUDA, "cost copy failed");
    if (parent && cudaMemcpy(parent, s->ds.gen_par, sizeof(int32_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_err(s, SPM_ERR_CUDA, "parent copy failed");
    return SPM_OK;
}

spm_status spm_scene_info(spm_scene *s, int64_t *info) {
    if (!s || !info) return set_err(s, SPM_ERR_INVALID_ARG, "null argument");
    int32_t stats[4] = {0, 0, 0, 0}, fc[4] = {0, 0, 1, 0};
    if (check_device(s) == SPM_OK) {
        cudaMemcpy(stats, s->ds.stats, sizeof stats, cudaMemcpyDeviceToHost);
        cudaMemcpy(fc, s->ds.flood_counts, sizeof fc, cudaMemcpyDeviceToHost);
    }
    info[0] = s->hs.n_gen;
    info[1] = s->hs.n_src;
    info[2] = s->hs.n_vert;
    info[3] = s->hs.S;
    info[4] = (int64_t)s->hs.poly_off.size() - 1;
    info[5] = stats[0];
    info[6] = stats[1];
    info[7] = s->ds.tile;
    info[8] = (s->ds.use_flood && fc[2] == 0) ? 1 : 0;
    info[9] = s->ds.flood_mode;
    const bool floods = s->ds.use_flood && s->ds.flood_mode != 2;
    // the geometric mode over kept obstacle-vertex lists: the sources' culling
    // (list reset, then the walk, or maps from every polygon and the tile
    // tests) and the list scan and fill
    const bool reuse = floods && s->ds.flood_mode == 3 && s->ds.static_tile_start;
    const int src_cull = !spm::flood_sources_direct(s->ds) ? 2 : s->ds.n_poly > 0 ? 3 : 2;
    // vertex phase (prep, pairs, edges, the tree's kernels, fixpoint kernels,
    // and after the many-CTA one its finalisation); flood, list scan and
    // fill; pixels
    const int many_cta = s->ds.fix_launch & (spm::kFixSoloSure | spm::kFixClusterSure) ? 0 : 2;
    info[10] = 1 + (s->hs.n_vert > 0 ? 4 : 0) + (s->ds.warm && s->ds.vtab ? 4 : 0) + (s->ds.fix_launch & spm::kFixSolo ? 1 : 0) +
               (s->ds.fix_launch & spm::kFixCluster ? 1 : 0) + many_cta + (floods ? (reuse ? src_cull + 2 : 3) : 0) + 1;
    return SPM_OK;
}

spm_status spm_scene_get_tuning(const spm_scene *s, spm_tuning *out) {
    if (!s || !out) return SPM_ERR_INVALID_ARG;
    *out = spm_tuning{};
    out->flood_mode = s->ds.flood_mode;
    out->hidden_chunk = s->ds.hidden_chunk;
    out->tile = s->ds.tile;
    out->maps = s->ds.use_maps;
    out->fixpoint_start = s->fix_start;
    return SPM_OK;
}

spm_status spm_scene_set_tuning(spm_scene *s, const spm_tuning *t) {
    if (!s || !t) return set_err(s, SPM_ERR_INVALID_ARG, "null argument");
    if (t->flood_mode < 0 || t->flood_mode > 3 || t->hidden_chunk < 32 || t->hidden_chunk > 256 ||
        (t->tile != 0 && t->tile != spm::kTile && t->tile != spm::kTileSmall) || t->maps < 0 || t->maps > 1 ||
        t->fixpoint_start < 0 || t->fixpoint_start > 2)
        return set_err(s, SPM_ERR_INVALID_ARG, "tuning out of range");
    s->fix_start = t->fixpoint_start;
    s->ds.warm = s->ds.vtab && (t->fixpoint_start == 2 || (t->fixpoint_start == 0 && s->warm_deep)) ? 1 : 0;
    s->ds.flood_mode = t->flood_mode;
    s->ds.hidden_chunk = t->hidden_chunk;
    s->ds.use_maps = t->maps && s->ds.gen_maps ? 1 : 0;
    if (t->tile) set_tile(s->ds, t->tile);
    return SPM_OK;
}

spm_status spm_scene_autotune(spm_scene *s, void *stream, spm_tuning *chosen) {
    if (!s) return set_err(nullptr, SPM_ERR_INVALID_ARG, "null scene");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    st = ensure_stage(s);
    if (st != SPM_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return set_err(s, SPM_ERR_CUDA, "event creation failed");
    const int modes[3] = {1, 2, 3}, chunks[2] = {32, 256}, tiles[2] = {spm::kTileSmall, spm::kTile};
    float best = 3.4e38f;
    spm_tuning pick{};
    pick.flood_mode = s->ds.flood_mode;
    pick.hidden_chunk = s->ds.hidden_chunk;
    pick.tile = s->ds.tile;
    pick.maps = s->ds.use_maps;
    pick.fixpoint_start = s->fix_start;
    for (int ui = 0; ui < 2; ++ui)
    for (int ti = 0; ti < 2; ++ti)
    for (int mi = 0; mi < 3; ++mi) {
        if (modes[mi] != 2 && !s->ds.use_flood) continue;
        if (ui == 1 && (modes[mi] == 2 || !s->ds.gen_maps)) continue;  // maps need a flood
        for (int ci = 0; ci < 2; ++ci) {
            s->ds.flood_mode = modes[mi];
            s->ds.hidden_chunk = chunks[ci];
            s->ds.use_maps = ui;
            set_tile(s->ds, tiles[ti]);
            float t[3];
            st = spm_compute(s, stream, s->stage_dist, s->stage_par);  // warm-up
            for (int k = 0; k < 3 && st == SPM_OK; ++k) {
                cudaEventRecord(a, cs);
                st = spm_compute(s, stream, s->stage_dist, s->stage_par);
                cudaEventRecord(b, cs);
                cudaEventSynchronize(b);
                cudaEventElapsedTime(&t[k], a, b);
            }
            if (st != SPM_OK) break;
            std::sort(t, t + 3);
            if (t[1] < best) {
                best = t[1];
                pick.flood_mode = modes[mi];
                pick.hidden_chunk = chunks[ci];
                pick.tile = tiles[ti];
                pick.maps = ui;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    s->ds.flood_mode = pick.flood_mode;
    s->ds.hidden_chunk = pick.hidden_chunk;
    s->ds.use_maps = pick.maps;
    set_tile(s->ds, pick.tile);
    if (chosen) *chosen = pick;
    if (st != SPM_OK) return st;
    return spm_scene_sync(s, stream);
}

spm_status spm_scene_phase_ms(spm_scene *s, float *vertex_ms, float *cull_ms, float *pixel_ms) {
    if (!s || !vertex_ms || !cull_ms || !pixel_ms) return set_err(s, SPM_ERR_INVALID_ARG, "null argument");
    if (!s->ev_valid) return set_err(s, SPM_ERR_INVALID_ARG, "no timed compute recorded");
    if (cudaEventSynchronize(s->ev[2]) != cudaSuccess ||
        cudaEventElapsedTime(vertex_ms, s->ev[0], s->ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(cull_ms, s->ev[1], s->ev[3]) != cudaSuccess ||
        cudaEventElapsedTime(pixel_ms, s->ev[3], s->ev[2]) != cudaSuccess)
        return set_err(s, SPM_ERR_CUDA, "event timing failed");
    return SPM_OK;
}

// Tape of the differentiable form: per agent its first gradient component
// (int32) and up to four values (float4), as two arrays.
static size_t tape_slot_bytes(int32_t n) { return ((size_t)n * sizeof(int32_t) + 15) & ~(size_t)15; }

int64_t spm_agents_tape_bytes(int32_t n) {
    return n < 0 ? 0 : (int64_t)(tape_slot_bytes(n) + (size_t)n * sizeof(float4));
}

spm_status spm_agents_forward(spm_scene *s, void *stream, const int32_t *agents_dev, int32_t n,
                              const float *dist_dev, const int32_t *parent_dev, float *loss_dev, void *tape_dev) {
    if (!s || (n > 0 && !agents_dev) || n < 0 || !dist_dev || !loss_dev || (tape_dev && !parent_dev))
        return set_err(s, SPM_ERR_INVALID_ARG, "bad argument");
    if (tape_dev && (reinterpret_cast<uintptr_t>(tape_dev) & 15))
        return set_err(s, SPM_ERR_INVALID_ARG, "tape must be 16-byte aligned");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    spm::launch_agents_forward(s->ds, cs, agents_dev, n, dist_dev, loss_dev, s->loss_partial);
    if (tape_dev) {
        unsigned char *t = static_cast<unsigned char *>(tape_dev);
        spm::launch_agents_contrib(s->ds, cs, agents_dev, n, parent_dev, s->root, s->lastpt,
                                   reinterpret_cast<int32_t *>(t), reinterpret_cast<float4 *>(t + tape_slot_bytes(n)));
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPM_OK : set_err(s, SPM_ERR_CUDA, cudaGetErrorString(e));
}

spm_status spm_agents_backward(spm_scene *s, void *stream, const void *tape_dev, int32_t n, float *grad_points_dev,
                               float *grad_segs_dev) {
    if (!s || n < 0 || (n > 0 && !tape_dev)) return set_err(s, SPM_ERR_INVALID_ARG, "bad argument");
    if ((s->hs.points.size() && !grad_points_dev) || (s->hs.segs.size() && !grad_segs_dev))
        return set_err(s, SPM_ERR_INVALID_ARG, "null gradient buffer");
    spm_status st = check_device(s);
    if (st != SPM_OK) return st;
    const unsigned char *t = static_cast<const unsigned char *>(tape_dev);
    spm::launch_agents_reduce((int)s->hs.points.size() / 2, (int)s->hs.segs.size() / 4,
                              static_cast<cudaStream_t>(stream), reinterpret_cast<const int32_t *>(t),
                              reinterpret_cast<const float4 *>(t + tape_slot_bytes(n)), n, s->grad_partial,
                              grad_points_dev, grad_segs_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPM_OK : set_err(s, SPM_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"

// Internal accessors for entry points defined in other translation units.
namespace spm {
const DevScene *scene_dev(const spm_scene *s) { return &s->ds; }
int scene_device(const spm_scene *s) { return s->device; }
void scene_set_error(spm_scene *s, const char *msg) { s->err = msg; }
}  // namespace spm
