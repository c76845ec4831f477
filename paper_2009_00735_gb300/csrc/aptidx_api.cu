// aptidx_api.cu -- the C ABI (include/aptidx.h): argument checks, ownership of
// device buffers, and the order of the launches of the hot path.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <mutex>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace aptidx {

int set_error(Ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

int cuda_check(Ctx* c, cudaError_t e, const char* what) {
    int code = (e == cudaErrorMemoryAllocation) ? APTIDX_E_OOM : APTIDX_E_CUDA;
    return set_error(c, code, "%s: %s", what, cudaGetErrorString(e));
}

constexpr size_t kSpareBytes = (size_t)4 << 30;

// sizes of the live blocks dev_alloc returned (all contexts; dev_free and
// release_spare drop them)
static std::mutex g_blk_mu;
static std::unordered_map<void*, size_t> g_blk_bytes;

int dev_alloc(Ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    for (size_t i = c->spare.size(); i-- > 0;) {
        if (c->spare[i].second == bytes) {
            *p = c->spare[i].first;
            c->spare_bytes -= bytes;
            c->spare.erase(c->spare.begin() + (ptrdiff_t)i);
            return APTIDX_OK;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation && !c->spare.empty()) {
        cudaGetLastError();
        release_spare(c);
        e = cudaMalloc(p, bytes);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(c, e == cudaErrorMemoryAllocation ? APTIDX_E_OOM : APTIDX_E_CUDA,
                         "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lk(g_blk_mu);
        g_blk_bytes[*p] = bytes;
    }
    return APTIDX_OK;
}

void dev_free(void* p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_blk_mu);
        g_blk_bytes.erase(p);
    }
    cudaFree(p);
}

void dev_recycle(Ctx* c, void* p) {
    if (!p) return;
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> lk(g_blk_mu);
        auto it = g_blk_bytes.find(p);
        if (it != g_blk_bytes.end()) bytes = it->second;
    }
    if (bytes == 0 || c->spare_bytes + bytes > kSpareBytes) {
        dev_free(p);
        return;
    }
    c->spare.emplace_back(p, bytes);
    c->spare_bytes += bytes;
}

void release_spare(Ctx* c) {
    for (auto& b : c->spare) dev_free(b.first);
    c->spare.clear();
    c->spare_bytes = 0;
}

template <typename T>
static void free_ptr(T*& p) {
    dev_free((void*)p);
    p = nullptr;
}

template <typename T>
static void recycle_ptr(Ctx* c, T*& p) {
    dev_recycle(c, (void*)p);
    p = nullptr;
}

// A host view of an input array: the caller's pointer for host memory, a
// copy for device memory.
template <typename T>
struct HostView {
    const T* p = nullptr;
    std::vector<T> own;
    const T& operator[](size_t i) const { return p[i]; }
    const T* data() const { return p; }
};

template <typename T>
static int to_host(Ctx* c, const T* src, size_t count, int mem, HostView<T>& out) {
    if (mem == APTIDX_MEM_HOST || count == 0) {
        out.p = src;
        return APTIDX_OK;
    }
    out.own.resize(count);
    APTIDX_CUDA(c, cudaMemcpyAsync(out.own.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
    out.p = out.own.data();
    return APTIDX_OK;
}

void prof_begin(Ctx* c, int phase) {
    if (!c->prof) return;
    cudaEvent_t e;
    if (!c->ev_pool.empty()) {
        e = c->ev_pool.back();
        c->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(e, c->stream);
    c->ev_open[phase] = e;
}

void prof_end(Ctx* c, int phase, int kernels) {
    c->launches += kernels;
    if (!c->prof || !c->ev_open[phase]) return;
    cudaEvent_t e;
    if (!c->ev_pool.empty()) {
        e = c->ev_pool.back();
        c->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(e, c->stream);
    c->ev_pending.push_back({phase, c->ev_open[phase], e});
    c->ev_open[phase] = nullptr;
}

static int check_mem(Ctx* c, int mem) {
    if (mem != APTIDX_MEM_HOST && mem != APTIDX_MEM_DEVICE)
        return set_error(c, APTIDX_E_INVALID_ARG, "mem must be APTIDX_MEM_HOST or APTIDX_MEM_DEVICE");
    return APTIDX_OK;
}

static int read_status(Ctx* c) {
    int st = 0;
    APTIDX_CUDA(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
    if (st) {
        APTIDX_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
        if (st & kStatusTimeout)
            return set_error(c, APTIDX_E_TIMEOUT, "a bounded device-side wait ran out (status 0x%x)", st);
        if (st & kStatusOverflow)
            return set_error(c, APTIDX_E_OVERFLOW, "a device-side count overflowed (status 0x%x)", st);
    }
    return APTIDX_OK;
}

static void clear_graphs(Ctx* c);

static void free_rois(Ctx* c) {
    clear_graphs(c);
    recycle_ptr(c, c->d_centres);
    recycle_ptr(c, c->d_radii);
    recycle_ptr(c, c->d_scale);
    recycle_ptr(c, c->d_band);
    recycle_ptr(c, c->d_nw);
    recycle_ptr(c, c->d_nw64);
    recycle_ptr(c, c->d_off);
    recycle_ptr(c, c->d_atoms);
    recycle_ptr(c, c->d_order);
    recycle_ptr(c, c->d_scan_tmp);
    c->nroi = 0;
    c->atoms_cap = c->atoms_total = 0;
    c->scan_tmp_elems = 0;
}

static void free_grid(Ctx* c) {
    recycle_ptr(c, c->d_cell_start);
    recycle_ptr(c, c->d_cell_pos);
    c->cell_h = 0.0;
    c->n_cells = 0;
}

static int ensure_scan_tmp(Ctx* c, int64_t n) {
    size_t need = scan_tmp_elems(n) + 1;
    if (c->scan_tmp_elems >= need) return APTIDX_OK;
    free_ptr(c->d_scan_tmp);
    int rc = dev_alloc(c, (void**)&c->d_scan_tmp, need * sizeof(int64_t));
    if (rc) return rc;
    c->scan_tmp_elems = need;
    return APTIDX_OK;
}

// Uniform cell grid with cell edge h over the positions' bounding box.
static int build_grid(Ctx* c, double h) {
    free_grid(c);
    int64_t n_cells = 1;
    for (;;) {
        n_cells = 1;
        for (int d = 0; d < 3; ++d) {
            double ext = c->hi[d] - c->lo[d];
            int dim = (int)std::max(1.0, ceil(ext / h));
            if (dim > (1 << 20)) dim = 1 << 20;
            c->dims[d] = dim;
            n_cells *= dim;
        }
        if (n_cells <= (int64_t)1 << 24) break;
        h *= 1.25;
    }
    c->cell_h = h;
    c->n_cells = n_cells;
    int rc;
    if ((rc = dev_alloc(c, (void**)&c->d_cell_start, (n_cells + 1) * sizeof(int64_t)))) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_cell_pos, c->n_atoms * sizeof(float4)))) return rc;
    const size_t nh = cell_sort_hist_elems(c->n_atoms);
    if ((rc = ensure_scan_tmp(c, std::max<int64_t>(n_cells, (int64_t)nh)))) return rc;
    int32_t *cell_of = nullptr, *k2 = nullptr, *idx = nullptr, *v2 = nullptr;
    int64_t *counts = nullptr, *hist = nullptr, *offs = nullptr;
    rc = dev_alloc(c, (void**)&cell_of, c->n_atoms * sizeof(int32_t));
    if (!rc) rc = dev_alloc(c, (void**)&k2, c->n_atoms * sizeof(int32_t));
    if (!rc) rc = dev_alloc(c, (void**)&idx, c->n_atoms * sizeof(int32_t));
    if (!rc) rc = dev_alloc(c, (void**)&v2, c->n_atoms * sizeof(int32_t));
    if (!rc) rc = dev_alloc(c, (void**)&counts, n_cells * sizeof(int64_t));
    if (!rc) rc = dev_alloc(c, (void**)&hist, nh * sizeof(int64_t));
    if (!rc) rc = dev_alloc(c, (void**)&offs, nh * sizeof(int64_t));
    if (!rc) {
        cudaError_t e = launch_cell_build(c, cell_of, k2, idx, v2, counts, hist, offs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = cuda_check(c, e, "cell grid build");
    }
    // the stream is synchronised above: the temporaries are idle
    dev_recycle(c, cell_of);
    dev_recycle(c, k2);
    dev_recycle(c, idx);
    dev_recycle(c, v2);
    dev_recycle(c, counts);
    dev_recycle(c, hist);
    dev_recycle(c, offs);
    if (rc) free_grid(c);
    return rc;
}

static void clear_graphs(Ctx* c) {
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

// gather count + offsets + fill (step a1), queued on the stream
static int run_gather(Ctx* c) {
    cudaError_t e = launch_gather_count(c);
    if (e == cudaSuccess) e = launch_gather_fill(c);
    if (e != cudaSuccess) return cuda_check(c, e, "ROI gather");
    return APTIDX_OK;
}

// The signature sequence of one compute call (a1-a5 and the optional
// normalisation), queued on the stream.
static int launch_sequence(Ctx* c, int path, unsigned flags, float* dS, uint16_t* dA) {
    int rc;
    prof_begin(c, APTIDX_PHASE_GATHER);
    if ((rc = run_gather(c))) return rc;
    prof_end(c, APTIDX_PHASE_GATHER, 6);
    prof_begin(c, APTIDX_PHASE_ORDER);
    cudaError_t e = launch_roi_order(c);
    if (e != cudaSuccess) return cuda_check(c, e, "ROI order");
    prof_end(c, APTIDX_PHASE_ORDER, 3);
    prof_begin(c, APTIDX_PHASE_SIGNATURE);
    if (path == APTIDX_PATH_PLAIN_FP32) {
        e = launch_signatures_plain(c, dS, dA, nullptr, -1, 0);
    } else {
        e = launch_signatures_tc(c, dS, dA, nullptr, -1);
    }
    if (e != cudaSuccess) return cuda_check(c, e, "signature kernel");
    prof_end(c, APTIDX_PHASE_SIGNATURE, path == APTIDX_PATH_PLAIN_FP32 ? 1 : 1);
    if (flags & APTIDX_NORMALISE_MAX) {
        prof_begin(c, APTIDX_PHASE_NORMALISE);
        e = launch_normalise(c, dS);
        if (e != cudaSuccess) return cuda_check(c, e, "normalise");
        prof_end(c, APTIDX_PHASE_NORMALISE, 1);
    }
    return APTIDX_OK;
}

// ---- autotuner ---------------------------------------------------------------
// Launch configuration per (path, bins, frequency groups of the band, mean
// ROI size, directions, device): tiles of 64 directions per work item and,
// on the tensor-core path, the number of MMA issuer warps.  Candidates are
// timed with CUDA events on the first ranks of the ROI order (8 per SM) and
// the fastest is kept for the context, and in the file named by the
// environment variable APTIDX_TUNE_CACHE when it is set.

static std::string tune_key(Ctx* c, int path) {
    char buf[384];
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, c->device);
    const double mean = c->nroi > 0 ? (double)c->atoms_total / (double)c->nroi : 0.0;
    const int abin = mean > 1.0 ? (int)lround(2.0 * log2(mean)) : 0;
    const int vbin = (int)lround(2.0 * log2((double)std::max(c->nv, 1)));
    const int groups = (c->band_max - c->band_min) / 4 + 1;
    const int pairs = c->use_pairs && c->npairs > 0 ? 1 : 0;
    snprintf(buf, sizeof(buf), "%s/%d|p%d|m%d|g%d|a%d|v%d|s%d", prop.name, prop.multiProcessorCount, path, c->m,
             groups, abin, vbin, pairs);
    for (char* q = buf; *q; ++q)
        if (*q == ' ') *q = '_';
    return buf;
}

static void tune_load(Ctx* c) {
    if (c->tune_loaded) return;
    c->tune_loaded = true;
    const char* path = getenv("APTIDX_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[200];
    int tpi, iss;
    float ms;
    while (fscanf(f, "%199s %d %d %f", key, &tpi, &iss, &ms) == 4) c->tune_cache[key] = {tpi, iss, ms};
    fclose(f);
}

static void tune_save(Ctx* c) {
    const char* path = getenv("APTIDX_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    for (auto& kv : c->tune_cache) fprintf(f, "%s %d %d %.4f\n", kv.first.c_str(), kv.second.tpi, kv.second.iss, kv.second.ms);
    fclose(f);
}

static int autotune(Ctx* c, int path, float* dS, uint16_t* dA) {
    tune_load(c);
    const int pi = path == APTIDX_PATH_TC_FP16 ? 1 : 0;
    const std::string key = tune_key(c, path);
    auto it = c->tune_cache.find(key);
    if (it != c->tune_cache.end()) {
        c->tune_tpi[pi] = it->second.tpi;
        if (pi) c->tune_iss = it->second.iss;
        return APTIDX_OK;
    }
    int rc;
    if ((rc = run_gather(c))) return rc;
    cudaError_t e = launch_roi_order(c);
    if (e != cudaSuccess) return cuda_check(c, e, "ROI order");
    const bool prof = c->prof;
    c->prof = false;
    c->rank_limit = std::min<int64_t>(c->nroi, (int64_t)8 * c->sm_count);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int tpis[] = {4, 8, 16, 32, 64};
    const int isss[] = {2, 4};
    Ctx::TuneCfg best{c->tune_tpi[pi], c->tune_iss, 1e30f};
    for (int tpi : tpis) {
        for (int iss : isss) {
            if (!pi && iss != 4) continue;
            c->tune_tpi[pi] = tpi;
            if (pi) c->tune_iss = iss;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first launch sets attributes
                e = cudaEventRecord(e0, c->stream);
                if (e == cudaSuccess)
                    e = pi ? launch_signatures_tc(c, dS, dA, nullptr, -1) : launch_signatures_plain(c, dS, dA, nullptr, -1, 0);
                if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            }
            if (e != cudaSuccess) break;
            if (ms < best.ms) best = {tpi, iss, ms};
        }
        if (e != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->rank_limit = 0;
    c->prof = prof;
    if (e != cudaSuccess) return cuda_check(c, e, "autotune");
    c->tune_tpi[pi] = best.tpi;
    if (pi) c->tune_iss = best.iss;
    c->tune_cache[key] = best;
    tune_save(c);
    return read_status(c);
}

}  // namespace aptidx

using namespace aptidx;

#define CTX_OR_FAIL(ctx)                                   \
    if (!(ctx)) return APTIDX_E_INVALID_ARG;               \
    Ctx* c = &(ctx)->c;                                    \
    c->err.clear();                                        \
    {                                                      \
        cudaError_t _e = cudaSetDevice(c->device);         \
        if (_e != cudaSuccess) return cuda_check(c, _e, "cudaSetDevice"); \
    }

extern "C" {

int aptidx_version(void) { return 100; }

int aptidx_band_for_spacing(double d_min, double d_max, double R, int m, int32_t* k_lo, int32_t* k_hi) {
    if (!k_lo || !k_hi) return APTIDX_E_INVALID_ARG;
    if (!(d_min > 0.0 && d_min <= d_max && isfinite(d_max))) return APTIDX_E_INVALID_ARG;
    if (!(R >= 1e-6 && R <= 1e6) || m < APTIDX_MIN_M || m > APTIDX_MAX_M) return APTIDX_E_INVALID_ARG;
    // W = 2^m dR = 2 (R + dR): the histogram span, whose k-th frequency bin has period W / k
    const double dR = R / (double)((1 << (m - 1)) - 1);
    const double W = 2.0 * (R + dR);
    const double lo = ceil(W / d_max), hi = floor(W / d_min);
    if (!(lo >= -2147483648.0 && hi <= 2147483647.0)) return APTIDX_E_INVALID_ARG;
    *k_lo = (int32_t)lo;
    *k_hi = (int32_t)hi;
    if (*k_lo < 0 || *k_hi < *k_lo || *k_hi > (1 << (m - 1))) return APTIDX_E_INVALID_ARG;
    return APTIDX_OK;
}

int aptidx_create(aptidx_ctx** out, int device, void* cuda_stream) {
    if (!out) return APTIDX_E_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return APTIDX_E_INVALID_ARG;
    }
    aptidx_ctx* h = new aptidx_ctx();
    Ctx* c = &h->c;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    int rc = APTIDX_OK;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) rc = APTIDX_E_CUDA;
    if (!rc) rc = dev_alloc(c, (void**)&c->d_status, sizeof(int) * 4);
    if (!rc) rc = dev_alloc(c, (void**)&c->d_counter, sizeof(int32_t) * 4);
    if (!rc) rc = dev_alloc(c, (void**)&c->d_sort_hist, sizeof(int32_t) * 65537);
    if (!rc && cudaMemsetAsync(c->d_status, 0, sizeof(int) * 4, c->stream) != cudaSuccess) rc = APTIDX_E_CUDA;
    if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = APTIDX_E_CUDA;
    if (rc) {
        aptidx_destroy(h);
        return rc;
    }
    *out = h;
    return APTIDX_OK;
}

int aptidx_destroy(aptidx_ctx* ctx) {
    if (!ctx) return APTIDX_E_INVALID_ARG;
    Ctx* c = &ctx->c;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_rois(c);
    free_grid(c);
    clear_graphs(c);
    free_ptr(c->d_S);
    free_ptr(c->d_argk);
    free_ptr(c->d_pos);
    free_ptr(c->d_types);
    free_ptr(c->d_dirs);
    free_ptr(c->d_dirs_sorted);
    free_ptr(c->d_slot_dirs);
    free_ptr(c->d_slot_idx);
    free_ptr(c->d_gn_scratch);
    c->gn_scratch_bytes = 0;
    free_ptr(c->d_match_scratch);
    c->match_scratch_bytes = 0;
    free_ptr(c->d_tw);
    dev_free(c->d_twb);
    c->d_twb = nullptr;
    free_ptr(c->d_status);
    free_ptr(c->d_counter);
    release_spare(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    free_ptr(c->d_sort_hist);
    for (auto& pr : c->ev_pending) {
        cudaEventDestroy(pr.a);
        cudaEventDestroy(pr.b);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (int i = 0; i < APTIDX_N_PHASES; ++i)
        if (c->ev_open[i]) cudaEventDestroy(c->ev_open[i]);
    for (int i = 0; i < kMaxCandidates; ++i) {
        Reference& r = c->ref[i];
        free_ptr(r.d_node_sig);
        free_ptr(r.d_top);
        free_ptr(r.d_top_val);
        free_ptr(r.d_img4);
        free_ptr(r.d_lut);
        free_ptr(r.d_quats);
    }
    delete ctx;
    return APTIDX_OK;
}

const char* aptidx_last_error(const aptidx_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->c.err.c_str();
}

int aptidx_sync(aptidx_ctx* ctx) {
    CTX_OR_FAIL(ctx);
    APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
    return read_status(c);
}

int aptidx_load_positions(aptidx_ctx* ctx, const float* xyz, int64_t n, const uint8_t* types, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if (!xyz || n <= 0 || n >= ((int64_t)1 << 31))
        return set_error(c, APTIDX_E_INVALID_ARG, "positions: need 0 < n < 2^31 and a non-NULL pointer");
    free_rois(c);
    free_grid(c);
    clear_graphs(c);
    c->n_atoms = 0;
    // a set of the same size reuses the device buffers (a reload per step
    // then costs the copy and the bounding box only)
    if (c->pos_cap != n) {
        free_ptr(c->d_pos);
        c->pos_cap = 0;
        if ((rc = dev_alloc(c, (void**)&c->d_pos, (size_t)n * 3 * sizeof(float)))) return rc;
        c->pos_cap = n;
    }
    const cudaMemcpyKind kind = mem == APTIDX_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    APTIDX_CUDA(c, cudaMemcpyAsync(c->d_pos, xyz, (size_t)n * 3 * sizeof(float), kind, c->stream));
    if (types) {
        if (c->types_cap != n) {
            free_ptr(c->d_types);
            c->types_cap = 0;
            if ((rc = dev_alloc(c, (void**)&c->d_types, (size_t)n))) return rc;
            c->types_cap = n;
        }
        APTIDX_CUDA(c, cudaMemcpyAsync(c->d_types, types, (size_t)n, kind, c->stream));
    } else {
        free_ptr(c->d_types);
        c->types_cap = 0;
    }
    // bounding box on the device; a NaN or infinite coordinate shows up as
    // a non-finite extreme (NaN patterns order beyond the infinities)
    float* mm = nullptr;
    if ((rc = dev_alloc(c, (void**)&mm, 12 * sizeof(float)))) return rc;
    cudaError_t e = launch_bbox(c->d_pos, n, mm, c->stream);
    float hmm[6];
    if (e == cudaSuccess) e = cudaMemcpyAsync(hmm, mm, sizeof(hmm), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(mm);
    if (e != cudaSuccess) return cuda_check(c, e, "bounding box");
    for (int d = 0; d < 6; ++d)
        if (!isfinite(hmm[d])) return set_error(c, APTIDX_E_INVALID_ARG, "positions: a coordinate is NaN or infinite");
    for (int d = 0; d < 3; ++d) {
        c->lo[d] = hmm[d];
        c->hi[d] = hmm[3 + d];
    }
    c->n_atoms = n;
    return APTIDX_OK;
}

int aptidx_set_directions(aptidx_ctx* ctx, const float* u, int32_t nv, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if (!u || nv <= 0) return set_error(c, APTIDX_E_INVALID_ARG, "directions: need nv > 0");
    HostView<float> hu;
    if ((rc = to_host(c, u, (size_t)nv * 3, mem, hu))) return rc;
    const int32_t nv_pad = (nv + kTileDirs - 1) / kTileDirs * kTileDirs;
    std::vector<float4> d4((size_t)nv_pad, make_float4(1.f, 0.f, 0.f, 0.f));
    for (int32_t v = 0; v < nv; ++v) {
        float x = hu[3 * v], y = hu[3 * v + 1], z = hu[3 * v + 2];
        double n2 = (double)x * x + (double)y * y + (double)z * z;
        if (!(fabs(sqrt(n2) - 1.0) <= 1e-5))
            return set_error(c, APTIDX_E_INVALID_ARG, "directions: |u[%d]| = %g is not 1", v, sqrt(n2));
        d4[v] = make_float4(x, y, z, 0.f);
    }
    // spatial order: Morton key of the (elevation, azimuth) 1-degree cell
    std::vector<std::pair<uint32_t, int32_t>> key((size_t)nv);
    for (int32_t v = 0; v < nv; ++v) {
        const double x = d4[v].x, y = d4[v].y, z = d4[v].z;
        const double el = asin(std::max(-1.0, std::min(1.0, z))) * (180.0 / M_PI) + 90.0;
        double az = atan2(y, x) * (180.0 / M_PI);
        if (az < 0.0) az += 360.0;
        const uint32_t i = (uint32_t)std::min(180.0, std::max(0.0, floor(el)));
        const uint32_t j = (uint32_t)std::min(359.0, std::max(0.0, floor(az)));
        uint32_t k = 0;
        for (int b = 0; b < 9; ++b) k |= ((i >> b) & 1u) << (2 * b + 1) | ((j >> b) & 1u) << (2 * b);
        key[v] = {k, v};
    }
    std::sort(key.begin(), key.end());
    std::vector<float4> ds((size_t)nv);
    for (int32_t k = 0; k < nv; ++k) {
        const int32_t v = key[k].second;
        int32_t bits = v;
        float w;
        memcpy(&w, &bits, sizeof(w));
        ds[k] = make_float4(d4[v].x, d4[v].y, d4[v].z, w);
    }
    // antipodal pairs: u_p = -u_v component by component (as values: a zero
    // of either sign matches), each direction in at most one pair; the lower
    // index is projected and writes its partner
    std::vector<std::tuple<uint32_t, uint32_t, uint32_t, int32_t>> keys((size_t)nv);
    auto zbits = [](float f) {
        const float g = f + 0.0f;   // -0 becomes +0
        uint32_t b;
        memcpy(&b, &g, sizeof(b));
        return b;
    };
    for (int32_t v = 0; v < nv; ++v) keys[v] = std::make_tuple(zbits(d4[v].x), zbits(d4[v].y), zbits(d4[v].z), v);
    std::sort(keys.begin(), keys.end());
    std::vector<int32_t> partner((size_t)nv, -1);
    int32_t npairs = 0;
    for (int32_t v = 0; v < nv; ++v) {
        if (partner[v] >= 0) continue;
        const auto want = std::make_tuple(zbits(-d4[v].x), zbits(-d4[v].y), zbits(-d4[v].z), (int32_t)-1);
        for (auto it = std::upper_bound(keys.begin(), keys.end(), want);
             it != keys.end() && std::get<0>(*it) == std::get<0>(want) && std::get<1>(*it) == std::get<1>(want) &&
             std::get<2>(*it) == std::get<2>(want);
             ++it) {
            const int32_t q = std::get<3>(*it);
            if (q != v && partner[q] < 0) {
                partner[v] = q;
                partner[q] = v;
                ++npairs;
                break;
            }
        }
    }
    std::vector<float4> sd;
    std::vector<int2> si;
    if (npairs > 0) {
        for (int32_t v = 0; v < nv; ++v) {
            if (partner[v] >= 0 && partner[v] < v) continue;   // written by its lower-index partner
            sd.push_back(d4[v]);
            si.push_back(make_int2(v, partner[v]));
        }
        while (sd.size() % kTileDirs) {
            sd.push_back(make_float4(1.f, 0.f, 0.f, 0.f));
            si.push_back(make_int2(-1, -1));
        }
    }
    free_ptr(c->d_dirs);
    free_ptr(c->d_dirs_sorted);
    free_ptr(c->d_slot_dirs);
    free_ptr(c->d_slot_idx);
    clear_graphs(c);
    c->nv = c->nv_pad = 0;
    c->nslot = c->nslot_pad = c->npairs = 0;
    if ((rc = dev_alloc(c, (void**)&c->d_dirs, (size_t)nv_pad * sizeof(float4)))) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_dirs_sorted, (size_t)nv * sizeof(float4)))) return rc;
    APTIDX_CUDA(c, cudaMemcpyAsync(c->d_dirs, d4.data(), (size_t)nv_pad * sizeof(float4), cudaMemcpyHostToDevice,
                                   c->stream));
    APTIDX_CUDA(c, cudaMemcpyAsync(c->d_dirs_sorted, ds.data(), (size_t)nv * sizeof(float4), cudaMemcpyHostToDevice,
                                   c->stream));
    if (npairs > 0) {
        if ((rc = dev_alloc(c, (void**)&c->d_slot_dirs, sd.size() * sizeof(float4)))) return rc;
        if ((rc = dev_alloc(c, (void**)&c->d_slot_idx, si.size() * sizeof(int2)))) return rc;
        APTIDX_CUDA(c, cudaMemcpyAsync(c->d_slot_dirs, sd.data(), sd.size() * sizeof(float4), cudaMemcpyHostToDevice,
                                       c->stream));
        APTIDX_CUDA(c, cudaMemcpyAsync(c->d_slot_idx, si.data(), si.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                       c->stream));
        c->nslot = nv - npairs;
        c->nslot_pad = (int32_t)sd.size();
        c->npairs = npairs;
    }
    APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
    c->nv = nv;
    c->nv_pad = nv_pad;
    for (int i = 0; i < kMaxCandidates; ++i) c->ref[i].nv_at_set = -1;   // references refer to old nodes
    return APTIDX_OK;
}

int aptidx_set_binning(aptidx_ctx* ctx, int m, int32_t k_lo, int32_t k_hi, int flags) {
    CTX_OR_FAIL(ctx);
    if (m < APTIDX_MIN_M || m > APTIDX_MAX_M)
        return set_error(c, APTIDX_E_INVALID_ARG, "m = %d outside [%d, %d]", m, APTIDX_MIN_M, APTIDX_MAX_M);
    if (k_lo < 0 || k_hi < k_lo || k_hi > (1 << (m - 1)))
        return set_error(c, APTIDX_E_INVALID_ARG, "band [%d, %d] outside [0, 2^(m-1)]", k_lo, k_hi);
    if (flags != 0) return set_error(c, APTIDX_E_INVALID_ARG, "flags must be 0");
    if (c->tw_m != m) {
        free_ptr(c->d_tw);
        c->tw_m = 0;
        int rc = dev_alloc(c, (void**)&c->d_tw, sizeof(float2) << m);
        if (rc) return rc;
        cudaError_t e = launch_twiddles(c->d_tw, m, c->stream);
        if (e != cudaSuccess) return cuda_check(c, e, "twiddles");
        c->tw_m = m;
    }
    if (c->m != m && c->nroi > 0) free_rois(c);   // per-ROI scales depend on m
    clear_graphs(c);
    c->m = m;
    c->k_lo = k_lo;
    c->k_hi = k_hi;
    c->binning_set = true;
    return APTIDX_OK;
}

int aptidx_set_rois(aptidx_ctx* ctx, const double* centres, const double* radii, int64_t nroi,
                    const int32_t* band_lo, const int32_t* band_hi, uint32_t type_mask, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if (c->n_atoms <= 0) return set_error(c, APTIDX_E_STATE, "set_rois: load positions first");
    if (c->nv <= 0) return set_error(c, APTIDX_E_STATE, "set_rois: set directions first");
    if (!c->binning_set) return set_error(c, APTIDX_E_STATE, "set_rois: set binning first");
    if (!centres || !radii || nroi <= 0 || nroi >= ((int64_t)1 << 30))
        return set_error(c, APTIDX_E_INVALID_ARG, "set_rois: need 0 < nroi < 2^30 and centres, radii");
    if ((band_lo == nullptr) != (band_hi == nullptr))
        return set_error(c, APTIDX_E_INVALID_ARG, "set_rois: band_lo and band_hi must both be given or both NULL");
    HostView<double> hc, hr;
    HostView<int32_t> hlo, hhi;
    if ((rc = to_host(c, centres, (size_t)nroi * 3, mem, hc))) return rc;
    if ((rc = to_host(c, radii, (size_t)nroi, mem, hr))) return rc;
    if (band_lo) {
        if ((rc = to_host(c, band_lo, (size_t)nroi, mem, hlo))) return rc;
        if ((rc = to_host(c, band_hi, (size_t)nroi, mem, hhi))) return rc;
    }
    const int half = 1 << (c->m - 1);
    std::vector<float> scale((size_t)nroi);
    std::vector<int32_t> band((size_t)nroi * 2);
    int32_t bmin = 1 << 30, bmax = -1;
    double rmax = 0.0;
    for (int64_t r = 0; r < nroi; ++r) {
        for (int d = 0; d < 3; ++d)
            if (!isfinite(hc[3 * r + d])) return set_error(c, APTIDX_E_INVALID_ARG, "centre %lld not finite", (long long)r);
        const double R = hr[r];
        if (!(R >= 1e-6 && R <= 1e6))
            return set_error(c, APTIDX_E_INVALID_ARG, "radius %lld must lie in [1e-6, 1e6] nm", (long long)r);
        scale[r] = (float)((double)(half - 1) / R);
        int32_t lo = band_lo ? hlo[r] : c->k_lo, hi = band_lo ? hhi[r] : c->k_hi;
        if (lo < 0 || hi < lo || hi > half)
            return set_error(c, APTIDX_E_INVALID_ARG, "band of ROI %lld [%d, %d] outside [0, %d]", (long long)r, lo, hi, half);
        band[2 * r] = lo;
        band[2 * r + 1] = hi;
        bmin = std::min(bmin, lo);
        bmax = std::max(bmax, hi);
        rmax = std::max(rmax, R);
    }
    free_rois(c);
    if ((rc = dev_alloc(c, (void**)&c->d_centres, (size_t)nroi * 3 * sizeof(double)))) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_radii, (size_t)nroi * sizeof(double)))) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_scale, (size_t)nroi * sizeof(float)))) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_band, (size_t)nroi * 2 * sizeof(int32_t)))) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_nw, (size_t)nroi * sizeof(int32_t)))) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_nw64, (size_t)nroi * sizeof(int64_t)))) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_off, (size_t)(nroi + 1) * sizeof(int64_t)))) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_order, (size_t)nroi * sizeof(int32_t)))) return rc;
    c->scan_tmp_elems = 0;
    if ((rc = ensure_scan_tmp(c, std::max<int64_t>(nroi, c->n_cells)))) return rc;
    cudaStream_t s = c->stream;
    APTIDX_CUDA(c, cudaMemcpyAsync(c->d_centres, hc.data(), (size_t)nroi * 3 * sizeof(double), cudaMemcpyHostToDevice, s));
    APTIDX_CUDA(c, cudaMemcpyAsync(c->d_radii, hr.data(), (size_t)nroi * sizeof(double), cudaMemcpyHostToDevice, s));
    APTIDX_CUDA(c, cudaMemcpyAsync(c->d_scale, scale.data(), scale.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    APTIDX_CUDA(c, cudaMemcpyAsync(c->d_band, band.data(), band.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    c->nroi = nroi;
    c->h_band = band;
    c->band_min = bmin;
    c->band_max = bmax;
    c->type_mask = type_mask;
    c->r_max = rmax;
    // cell grid sized for the largest ROI (edge ~ R_max / 2, at least 0.25 nm)
    const double want_h = std::max(rmax / 2.0, 0.25);
    if (c->cell_h <= 0.0 || c->cell_h < 0.7 * want_h || c->cell_h > 1.5 * want_h) {
        if ((rc = build_grid(c, want_h))) {
            free_rois(c);
            return rc;
        }
        if ((rc = ensure_scan_tmp(c, std::max<int64_t>(nroi, c->n_cells)))) return rc;
    }
    // count the ROI atoms once to size the gather buffer
    APTIDX_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
    cudaError_t e = launch_gather_count(c);
    if (e != cudaSuccess) return cuda_check(c, e, "ROI count");
    std::vector<int32_t> hnw((size_t)nroi);
    APTIDX_CUDA(c, cudaMemcpyAsync(hnw.data(), c->d_nw, (size_t)nroi * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    APTIDX_CUDA(c, cudaStreamSynchronize(s));
    int64_t total = 0;
    int32_t nwmax = 0;
    for (int64_t r = 0; r < nroi; ++r) {
        total += hnw[r];
        nwmax = std::max(nwmax, hnw[r]);
    }
    if (nwmax > APTIDX_MAX_ATOMS_PER_ROI) {
        APTIDX_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
        free_rois(c);
        return set_error(c, APTIDX_E_OVERFLOW, "a ROI holds %d selected atoms (limit %d)", nwmax,
                         APTIDX_MAX_ATOMS_PER_ROI);
    }
    c->nw_max = nwmax;
    c->atoms_total = total;
    c->atoms_cap = std::max<int64_t>(total, 1);
    if ((rc = dev_alloc(c, (void**)&c->d_atoms, (size_t)c->atoms_cap * sizeof(float4)))) return rc;
    return read_status(c);
}

int aptidx_compute_signatures(aptidx_ctx* ctx, int path, unsigned flags, float* S, uint16_t* argk,
                              int32_t* n_atoms, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if (c->nroi <= 0) return set_error(c, APTIDX_E_STATE, "compute_signatures: set ROIs first");
    if (path != APTIDX_PATH_PLAIN_FP32 && path != APTIDX_PATH_TC_FP16)
        return set_error(c, APTIDX_E_INVALID_ARG, "unknown path %d", path);
    if (flags & ~(APTIDX_NORMALISE_MAX | APTIDX_AUTOTUNE | APTIDX_GRAPH | APTIDX_DIRECT))
        return set_error(c, APTIDX_E_INVALID_ARG, "unknown flags 0x%x", flags);
    c->use_pairs = !(flags & APTIDX_DIRECT);
    const int64_t nS = c->nroi * (int64_t)c->nv;
    float* dS = S;
    uint16_t* dA = argk;
    if (mem == APTIDX_MEM_HOST || !S) {
        if (c->S_cap < nS) {
            free_ptr(c->d_S);
            free_ptr(c->d_argk);
            c->S_cap = 0;
            if ((rc = dev_alloc(c, (void**)&c->d_S, (size_t)nS * sizeof(float)))) return rc;
            if ((rc = dev_alloc(c, (void**)&c->d_argk, (size_t)nS * sizeof(uint16_t)))) return rc;
            c->S_cap = nS;
        }
        dS = c->d_S;
        dA = argk ? c->d_argk : nullptr;
    }
    if (path == APTIDX_PATH_TC_FP16 && (rc = prepare_tc(c))) return rc;
    if ((flags & APTIDX_AUTOTUNE) && (rc = autotune(c, path, dS, dA))) return rc;
    if (flags & APTIDX_GRAPH) {
        // capture the sequence once per (arguments, configuration), replay after
        char kb[256];
        snprintf(kb, sizeof(kb), "%d|%u|%p|%p|%lld|%d|%d|%d|%d", path, flags & (APTIDX_NORMALISE_MAX | APTIDX_DIRECT),
                 (void*)dS, (void*)dA,
                 (long long)c->nroi, c->nv, c->m, c->tune_tpi[path == APTIDX_PATH_TC_FP16], c->tune_iss);
        auto it = c->graphs.find(kb);
        if (it == c->graphs.end()) {
            // capture on a private stream (capture is not possible on the
            // legacy default stream); the graph then runs on the caller's stream
            if (!c->cap_stream) APTIDX_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
            const bool prof = c->prof;
            c->prof = false;
            const int64_t l0 = c->launches;
            cudaStream_t user = c->stream;
            cudaGraph_t g = nullptr;
            APTIDX_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            c->stream = c->cap_stream;
            rc = launch_sequence(c, path, flags, dS, dA);
            c->stream = user;
            cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
            c->prof = prof;
            c->launches = l0;
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return cuda_check(c, e, "graph capture");
            cudaGraphExec_t x = nullptr;
            e = cudaGraphInstantiate(&x, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_check(c, e, "graph instantiate");
            it = c->graphs.emplace(kb, x).first;
        }
        prof_begin(c, APTIDX_PHASE_SIGNATURE);
        APTIDX_CUDA(c, cudaGraphLaunch(it->second, c->stream));
        prof_end(c, APTIDX_PHASE_SIGNATURE, (path == APTIDX_PATH_TC_FP16 ? 11 : 10) + ((flags & APTIDX_NORMALISE_MAX) ? 1 : 0));
    } else if ((rc = launch_sequence(c, path, flags, dS, dA))) {
        return rc;
    }
    c->use_pairs = true;
    if (mem == APTIDX_MEM_HOST) {
        if (S) APTIDX_CUDA(c, cudaMemcpyAsync(S, dS, (size_t)nS * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        if (argk)
            APTIDX_CUDA(c, cudaMemcpyAsync(argk, dA, (size_t)nS * sizeof(uint16_t), cudaMemcpyDeviceToHost, c->stream));
        if (n_atoms)
            APTIDX_CUDA(c, cudaMemcpyAsync(n_atoms, c->d_nw, (size_t)c->nroi * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                           c->stream));
        return read_status(c);
    }
    if (n_atoms)
        APTIDX_CUDA(c, cudaMemcpyAsync(n_atoms, c->d_nw, (size_t)c->nroi * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                       c->stream));
    return APTIDX_OK;
}

int aptidx_path_supported(aptidx_ctx* ctx, int path) {
    if (!ctx) return 0;
    if (path == APTIDX_PATH_PLAIN_FP32) return 1;
    if (path == APTIDX_PATH_TC_FP16) return tc_supported(&ctx->c) ? 1 : 0;
    return 0;
}

int aptidx_get_tuning(aptidx_ctx* ctx, int path, int32_t* tiles_per_item, int32_t* issuers) {
    CTX_OR_FAIL(ctx);
    if (path != APTIDX_PATH_PLAIN_FP32 && path != APTIDX_PATH_TC_FP16)
        return set_error(c, APTIDX_E_INVALID_ARG, "unknown path %d", path);
    if (tiles_per_item) *tiles_per_item = c->tune_tpi[path == APTIDX_PATH_TC_FP16];
    if (issuers) *issuers = path == APTIDX_PATH_TC_FP16 ? c->tune_iss : 0;
    return APTIDX_OK;
}

namespace aptidx {
namespace {
// every thread streams 16-byte words of the buffer (grid-stride, four loads
// in flight), `iters` passes; the XOR of what it read keeps the loads alive
__global__ void __launch_bounds__(256) k_l2_read(const uint4* __restrict__ buf, int64_t n16, int iters,
                                                 uint32_t* sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
        int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(v[u].x), "=r"(v[u].y), "=r"(v[u].z), "=r"(v[u].w)
                             : "l"(buf + i + u * stride));
#pragma unroll
            for (int u = 0; u < 4; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        }
        for (; i < n16; i += stride) {
            uint4 v;
            asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                         : "l"(buf + i));
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    if (acc == 0x9E3779B9u) *sink = acc;
}

// Every lane adds 1 to words of its own bank (lane l: word l of a 128-byte
// row) of a 1024-row shared array, as the signature histograms do; the rows
// are drawn once per lane (16 of them, from a 32-bit mixing hash) and XORed
// with the step number, so consecutive increments of a lane land in
// different rows.  Block b writes the sum of its array (which must equal
// threads x iters x 16) to sums[b] and its clock64 cycles to cycles[b].
__global__ void __launch_bounds__(1024) k_smem_red(int iters, uint32_t* sums, long long* cycles) {
    extern __shared__ __align__(16) uint32_t sh[];   // [1024][32]
    for (int i = threadIdx.x; i < 1024 * 32; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(sh) + 4u * (threadIdx.x & 31u);
    uint32_t a[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        uint32_t h = (blockIdx.x * blockDim.x + threadIdx.x) * 16u + (uint32_t)u + 0x9E3779B9u;
        h ^= h >> 16;
        h *= 0x7FEB352Du;
        h ^= h >> 15;
        h *= 0x846CA68Bu;
        h ^= h >> 16;
        a[u] = base + (h >> 22) * 128u;
    }
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
        const uint32_t x = ((uint32_t)it & 1023u) * 128u;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const uint32_t ad = (a[u] - base) ^ x;
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(base + ad), "r"(1u) : "memory");
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t part = 0;
    for (int i = threadIdx.x; i < 1024 * 32; i += blockDim.x) part += sh[i];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
        sums[blockIdx.x] = tot;
        cycles[blockIdx.x] = t1 - t0;
    }
}
}  // namespace
}  // namespace aptidx

int aptidx_probe_l2(aptidx_ctx* ctx, int64_t bytes, int32_t iters, double* gbs) {
    CTX_OR_FAIL(ctx);
    if (bytes < (1 << 20) || bytes > ((int64_t)96 << 20) || bytes % 16 != 0 || iters < 1 || iters > 100000 || !gbs)
        return set_error(c, APTIDX_E_INVALID_ARG, "probe_l2: bytes in [1 MiB, 96 MiB], a multiple of 16; iters >= 1");
    void* buf = nullptr;
    int rc = dev_alloc(c, &buf, (size_t)bytes + 256);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemsetAsync(buf, 1, (size_t)bytes + 256, c->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const unsigned grid = (unsigned)c->sm_count * 8;
    const uint4* b16 = static_cast<const uint4*>(buf);
    uint32_t* sink = reinterpret_cast<uint32_t*>(static_cast<char*>(buf) + bytes);
    if (e == cudaSuccess) {
        k_l2_read<<<grid, 256, 0, c->stream>>>(b16, bytes / 16, 1, sink);   // brings the buffer into L2
        e = cudaEventRecord(e0, c->stream);
    }
    if (e == cudaSuccess) {
        k_l2_read<<<grid, 256, 0, c->stream>>>(b16, bytes / 16, iters, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(buf);
    if (e != cudaSuccess) return cuda_check(c, e, "probe_l2");
    c->launches += 2;
    *gbs = (double)bytes * iters / (ms * 1e-3) / 1e9;
    return APTIDX_OK;
}

int aptidx_probe_smem_atomics(aptidx_ctx* ctx, int32_t threads, int32_t iters, double* incr_per_s,
                              double* reds_per_sm_cycle) {
    CTX_OR_FAIL(ctx);
    if (threads < 32 || threads > 1024 || threads % 32 != 0 || iters < 1 || iters > 1000000 || !incr_per_s)
        return set_error(c, APTIDX_E_INVALID_ARG,
                         "probe_smem_atomics: threads a multiple of 32 in [32, 1024], iters in [1, 1e6]");
    const int nb = c->sm_count;
    void* buf = nullptr;
    int rc = dev_alloc(c, &buf, (size_t)nb * 12 + 64);
    if (rc) return rc;
    long long* cyc = static_cast<long long*>(buf);
    uint32_t* sums = reinterpret_cast<uint32_t*>(cyc + nb);
    const size_t smem = 1024 * 128;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaFuncSetAttribute(k_smem_red, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_smem_red<<<nb, threads, smem, c->stream>>>(1, sums, cyc);   // warm-up
        e = cudaEventRecord(e0, c->stream);
    }
    if (e == cudaSuccess) {
        k_smem_red<<<nb, threads, smem, c->stream>>>(iters, sums, cyc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    std::vector<long long> hc(nb);
    std::vector<uint32_t> hs(nb);
    if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, (size_t)nb * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hs.data(), sums, (size_t)nb * 4, cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(buf);
    if (e != cudaSuccess) return cuda_check(c, e, "probe_smem_atomics");
    c->launches += 2;
    const uint32_t want = (uint32_t)((uint64_t)threads * (uint64_t)iters * 16u);
    double cyc_mean = 0.0;
    for (int b = 0; b < nb; ++b) {
        if (hs[b] != want)
            return set_error(c, APTIDX_E_CUDA, "probe_smem_atomics: block %d counted %u increments, expected %u", b,
                             hs[b], want);
        cyc_mean += (double)hc[b] / nb;
    }
    const double incr = (double)nb * threads * (double)iters * 16.0;
    *incr_per_s = incr / (ms * 1e-3);
    if (reds_per_sm_cycle) *reds_per_sm_cycle = (double)threads / 32.0 * iters * 16.0 / cyc_mean;
    return APTIDX_OK;
}

int aptidx_set_profiling(aptidx_ctx* ctx, int enable) {
    CTX_OR_FAIL(ctx);
    APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto& pr : c->ev_pending) {
        c->ev_pool.push_back(pr.a);
        c->ev_pool.push_back(pr.b);
    }
    c->ev_pending.clear();
    for (int i = 0; i < APTIDX_N_PHASES; ++i) {
        if (c->ev_open[i]) c->ev_pool.push_back(c->ev_open[i]);
        c->ev_open[i] = nullptr;
        c->prof_ms[i] = 0.0;
        c->prof_calls[i] = 0;
    }
    c->launches = 0;
    c->prof = enable != 0;
    return APTIDX_OK;
}

int aptidx_get_profile(aptidx_ctx* ctx, double* phase_ms, int64_t* phase_calls, int64_t* launches) {
    CTX_OR_FAIL(ctx);
    APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto& pr : c->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pr.a, pr.b) == cudaSuccess) {
            c->prof_ms[pr.phase] += ms;
            c->prof_calls[pr.phase] += 1;
        } else {
            cudaGetLastError();
        }
        c->ev_pool.push_back(pr.a);
        c->ev_pool.push_back(pr.b);
    }
    c->ev_pending.clear();
    for (int i = 0; i < APTIDX_N_PHASES; ++i) {
        if (phase_ms) phase_ms[i] = c->prof_ms[i];
        if (phase_calls) phase_calls[i] = c->prof_calls[i];
    }
    if (launches) *launches = c->launches;
    return APTIDX_OK;
}

int aptidx_get_histograms(aptidx_ctx* ctx, int64_t roi, int path, uint16_t* h, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if (c->nroi <= 0) return set_error(c, APTIDX_E_STATE, "get_histograms: set ROIs first");
    if (roi < 0 || roi >= c->nroi || !h) return set_error(c, APTIDX_E_INVALID_ARG, "get_histograms: bad roi or NULL h");
    if (path != APTIDX_PATH_PLAIN_FP32 && path != APTIDX_PATH_TC_FP16)
        return set_error(c, APTIDX_E_INVALID_ARG, "unknown path %d", path);
    const size_t n = (size_t)c->nv << c->m;
    uint16_t* dh = h;
    if (mem == APTIDX_MEM_HOST && (rc = dev_alloc(c, (void**)&dh, n * sizeof(uint16_t)))) return rc;
    // scratch signature row for the single ROI
    float* row = nullptr;
    if ((rc = dev_alloc(c, (void**)&row, (size_t)c->nv * sizeof(float)))) {
        if (mem == APTIDX_MEM_HOST) dev_free(dh);
        return rc;
    }
    rc = run_gather(c);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        // the kernels add the counts of every (atom block, bin chunk) pass
        e = cudaMemsetAsync(dh, 0, n * sizeof(uint16_t), c->stream);
        if (e != cudaSuccess) rc = cuda_check(c, e, "zero histograms");
    }
    if (!rc) {
        if (path == APTIDX_PATH_PLAIN_FP32) {
            e = launch_signatures_plain(c, row, nullptr, dh, roi, 0);
        } else {
            rc = prepare_tc(c);
            if (!rc) e = launch_signatures_tc(c, row, nullptr, dh, roi);
        }
        if (!rc && e != cudaSuccess) rc = cuda_check(c, e, "histogram export");
    }
    if (!rc && mem == APTIDX_MEM_HOST) {
        e = cudaMemcpyAsync(h, dh, n * sizeof(uint16_t), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) rc = cuda_check(c, e, "copy histograms");
    }
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (!rc && e2 != cudaSuccess) rc = cuda_check(c, e2, "sync");
    dev_free(row);
    if (mem == APTIDX_MEM_HOST) dev_free(dh);
    if (rc) return rc;
    return read_status(c);
}

int aptidx_get_roi_atoms(aptidx_ctx* ctx, int64_t roi, float* xc, int64_t cap, int64_t* n_out, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if (c->nroi <= 0) return set_error(c, APTIDX_E_STATE, "get_roi_atoms: set ROIs first");
    if (roi < 0 || roi >= c->nroi || !n_out) return set_error(c, APTIDX_E_INVALID_ARG, "get_roi_atoms: bad arguments");
    if ((rc = run_gather(c))) return rc;
    int64_t off[2];
    APTIDX_CUDA(c, cudaMemcpyAsync(off, c->d_off + roi, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
    const int64_t n = off[1] - off[0];
    *n_out = n;
    if (n > cap || (n > 0 && !xc)) return set_error(c, APTIDX_E_OVERFLOW, "get_roi_atoms: %lld atoms exceed cap %lld", (long long)n, (long long)cap);
    std::vector<float4> tmp((size_t)n);
    if (n > 0) {
        APTIDX_CUDA(c, cudaMemcpyAsync(tmp.data(), c->d_atoms + off[0], (size_t)n * sizeof(float4), cudaMemcpyDeviceToHost,
                                       c->stream));
        APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    std::vector<float> packed((size_t)n * 3);
    for (int64_t i = 0; i < n; ++i) {
        packed[3 * i] = tmp[i].x;
        packed[3 * i + 1] = tmp[i].y;
        packed[3 * i + 2] = tmp[i].z;
    }
    if (n > 0) {
        APTIDX_CUDA(c, cudaMemcpyAsync(xc, packed.data(), packed.size() * sizeof(float),
                                       mem == APTIDX_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice,
                                       c->stream));
        APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return read_status(c);
}

}  // extern "C"

// ---- indexing (a6) and refinement (a7) --------------------------------------

namespace {

// device buffer freed at scope exit
struct DevTmp {
    void* p = nullptr;
    ~DevTmp() { dev_free(p); }
};

// Device view of an input array: the pointer itself (device) or a temporary
// device copy (host).
template <typename T>
int dev_view(Ctx* c, const T* src, size_t count, int mem, DevTmp& tmp, const T** out) {
    if (mem == APTIDX_MEM_DEVICE || count == 0) {
        *out = src;
        return APTIDX_OK;
    }
    int rc = dev_alloc(c, &tmp.p, count * sizeof(T));
    if (rc) return rc;
    APTIDX_CUDA(c, cudaMemcpyAsync(tmp.p, src, count * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    *out = static_cast<const T*>(tmp.p);
    return APTIDX_OK;
}

// Device destination of an output: the pointer itself (device) or a
// temporary to copy back after the launch (host).
template <typename T>
int dev_out(Ctx* c, T* dst, size_t count, int mem, DevTmp& tmp, T** out) {
    if (!dst || mem == APTIDX_MEM_DEVICE) {
        *out = dst;
        return APTIDX_OK;
    }
    int rc = dev_alloc(c, &tmp.p, count * sizeof(T));
    if (rc) return rc;
    *out = static_cast<T*>(tmp.p);
    return APTIDX_OK;
}

template <typename T>
int copy_back(Ctx* c, T* dst, const T* dsrc, size_t count, int mem) {
    if (!dst || mem == APTIDX_MEM_DEVICE) return APTIDX_OK;
    APTIDX_CUDA(c, cudaMemcpyAsync(dst, dsrc, count * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    return APTIDX_OK;
}

int check_ref(Ctx* c, int32_t cand, bool need_lut, bool need_img) {
    if (cand < 0 || cand >= kMaxCandidates) return set_error(c, APTIDX_E_INVALID_ARG, "candidate %d outside [0, %d)", cand, kMaxCandidates);
    const Reference& r = c->ref[cand];
    if (!r.d_node_sig || r.nv_at_set != c->nv)
        return set_error(c, APTIDX_E_STATE, "candidate %d: set the reference for the current directions first", cand);
    if (need_lut && (!r.d_lut || r.ng <= 0)) return set_error(c, APTIDX_E_STATE, "candidate %d: build the look-up table first", cand);
    if (need_img && !r.d_img4) return set_error(c, APTIDX_E_STATE, "candidate %d: no reference image", cand);
    return APTIDX_OK;
}

}  // namespace

extern "C" {

int aptidx_set_reference(aptidx_ctx* ctx, int32_t cand, const float* node_sig, int32_t n_hat, const float* img, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if (cand < 0 || cand >= kMaxCandidates) return set_error(c, APTIDX_E_INVALID_ARG, "candidate %d outside [0, %d)", cand, kMaxCandidates);
    if (c->nv <= 0) return set_error(c, APTIDX_E_STATE, "set_reference: set directions first");
    if (!node_sig || n_hat < 1 || n_hat > c->nv)
        return set_error(c, APTIDX_E_INVALID_ARG, "set_reference: need node_sig and 1 <= n_hat <= nv");
    HostView<float> hs;
    if ((rc = to_host(c, node_sig, (size_t)c->nv, mem, hs))) return rc;
    for (int32_t v = 0; v < c->nv; ++v)
        if (!isfinite(hs[v])) return set_error(c, APTIDX_E_INVALID_ARG, "set_reference: node value %d not finite", v);
    Reference& r = c->ref[cand];
    free_ptr(r.d_node_sig);
    free_ptr(r.d_top);
    free_ptr(r.d_top_val);
    free_ptr(r.d_lut);
    free_ptr(r.d_quats);
    free_ptr(r.d_img4);
    r.ng = 0;
    r.nv_at_set = -1;
    if ((rc = dev_alloc(c, (void**)&r.d_node_sig, (size_t)c->nv * sizeof(float)))) return rc;
    if ((rc = dev_alloc(c, (void**)&r.d_top, (size_t)n_hat * sizeof(int32_t)))) return rc;
    if ((rc = dev_alloc(c, (void**)&r.d_top_val, (size_t)n_hat * sizeof(float)))) return rc;
    APTIDX_CUDA(c, cudaMemcpyAsync(r.d_node_sig, hs.data(), (size_t)c->nv * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    if (img) {
        HostView<float> hi;
        const size_t ni = (size_t)kImgRows * kImgCols;
        if ((rc = to_host(c, img, ni, mem, hi))) return rc;
        for (size_t i = 0; i < ni; ++i)
            if (!isfinite(hi[i])) return set_error(c, APTIDX_E_INVALID_ARG, "set_reference: image value %zu not finite", i);
        // the four taps of every bilinear cell side by side: one 16-byte read
        // per sample
        const size_t nc = (size_t)(kImgRows - 1) * kImgCols;
        std::vector<float4> cells(nc);
        for (int i = 0; i + 1 < kImgRows; ++i)
            for (int j = 0; j < kImgCols; ++j) {
                const int j1 = j + 1 == kImgCols ? 0 : j + 1;
                cells[(size_t)i * kImgCols + j] =
                    make_float4(hi[(size_t)i * kImgCols + j], hi[(size_t)i * kImgCols + j1],
                                hi[(size_t)(i + 1) * kImgCols + j], hi[(size_t)(i + 1) * kImgCols + j1]);
            }
        if ((rc = dev_alloc(c, (void**)&r.d_img4, nc * sizeof(float4)))) return rc;
        APTIDX_CUDA(c, cudaMemcpyAsync(r.d_img4, cells.data(), nc * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
        APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));   // `cells` is released on return
    }
    r.n_hat = n_hat;
    {
        // energy of the strongest n_hat values (which nodes tie at the cut does
        // not change it), FP64
        std::vector<float> v(hs.data(), hs.data() + c->nv);
        std::nth_element(v.begin(), v.begin() + (n_hat - 1), v.end(), std::greater<float>());
        double en = 0.0;
        for (int32_t k = 0; k < n_hat; ++k) en += (double)v[k] * (double)v[k];
        r.energy = en;
    }
    cudaError_t e = launch_top_nodes(c, &r);
    if (e != cudaSuccess) return cuda_check(c, e, "strongest reference nodes");
    c->launches += 1;
    r.nv_at_set = c->nv;
    return APTIDX_OK;
}

int aptidx_build_lut(aptidx_ctx* ctx, int32_t cand, const double* quats, int64_t ng, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if ((rc = check_ref(c, cand, false, false))) return rc;
    if (!quats || ng <= 0 || ng > ((int64_t)1 << 31) / std::max(1, c->ref[cand].n_hat))
        return set_error(c, APTIDX_E_INVALID_ARG, "build_lut: need quats and 0 < ng * n_hat < 2^31");
    HostView<double> hq;
    if ((rc = to_host(c, quats, (size_t)ng * 4, mem, hq))) return rc;
    for (int64_t g = 0; g < ng; ++g) {
        const double n = sqrt(hq[4 * g] * hq[4 * g] + hq[4 * g + 1] * hq[4 * g + 1] + hq[4 * g + 2] * hq[4 * g + 2] +
                              hq[4 * g + 3] * hq[4 * g + 3]);
        if (!(fabs(n - 1.0) <= 1e-6)) return set_error(c, APTIDX_E_INVALID_ARG, "build_lut: quaternion %lld not unit", (long long)g);
    }
    Reference& r = c->ref[cand];
    free_ptr(r.d_lut);
    free_ptr(r.d_quats);
    r.ng = 0;
    r.ng_pad = 0;
    if ((rc = dev_alloc(c, (void**)&r.d_quats, (size_t)ng * 4 * sizeof(double)))) return rc;
    APTIDX_CUDA(c, cudaMemcpyAsync(r.d_quats, hq.data(), (size_t)ng * 4 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    r.ng_pad = (ng + 7) / 8 * 8;
    r.lut_bytes = c->nv <= 65536 ? 2 : 4;
    if ((rc = dev_alloc(c, &r.d_lut, (size_t)r.ng_pad * r.n_hat * r.lut_bytes))) return rc;
    APTIDX_CUDA(c, cudaMemsetAsync(r.d_lut, 0, (size_t)r.ng_pad * r.n_hat * r.lut_bytes, c->stream));
    cudaError_t e = launch_build_lut(c, &r, r.d_quats, ng);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "look-up table");
    c->launches += 1;
    r.ng = ng;
    return APTIDX_OK;
}

int aptidx_get_lut(aptidx_ctx* ctx, int32_t cand, int32_t* lut, int32_t* n_hat_out, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if ((rc = check_ref(c, cand, true, false))) return rc;
    Reference& r = c->ref[cand];
    if (n_hat_out) *n_hat_out = r.n_hat;
    if (!lut) return APTIDX_OK;
    DevTmp t;
    int32_t* d;
    const size_t n = (size_t)r.ng * r.n_hat;
    if ((rc = dev_out(c, lut, n, mem, t, &d))) return rc;
    cudaError_t e = launch_lut_export(c, &r, d);
    if (e != cudaSuccess) return cuda_check(c, e, "look-up table export");
    if ((rc = copy_back(c, lut, d, n, mem))) return rc;
    APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
    return APTIDX_OK;
}

int aptidx_match(aptidx_ctx* ctx, int32_t cand, const float* S, int64_t nroi, int32_t* best, float* score, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if ((rc = check_ref(c, cand, true, false))) return rc;
    if (!S || !best || nroi <= 0) return set_error(c, APTIDX_E_INVALID_ARG, "match: need S, best and nroi > 0");
    Reference& r = c->ref[cand];
    static int max_optin = -1;
    if (max_optin < 0) cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (((size_t)c->nv + r.n_hat) * sizeof(float) > (size_t)max_optin)
        return set_error(c, APTIDX_E_INVALID_ARG, "match: %d directions do not fit one shared-memory signature row", c->nv);
    DevTmp tS, tb, ts;
    const float* dS;
    int32_t* db;
    float* ds;
    if ((rc = dev_view(c, S, (size_t)nroi * c->nv, mem, tS, &dS))) return rc;
    if ((rc = dev_out(c, best, (size_t)nroi, mem, tb, &db))) return rc;
    if ((rc = dev_out(c, score, (size_t)nroi, mem, ts, &ds))) return rc;
    prof_begin(c, APTIDX_PHASE_MATCH);
    cudaError_t e = launch_match(c, &r, dS, nroi, db, ds);
    if (e != cudaSuccess) return cuda_check(c, e, "match");
    prof_end(c, APTIDX_PHASE_MATCH, 1);
    if ((rc = copy_back(c, best, db, (size_t)nroi, mem))) return rc;
    if ((rc = copy_back(c, score, ds, (size_t)nroi, mem))) return rc;
    if (mem == APTIDX_MEM_HOST) return read_status(c);
    return APTIDX_OK;
}

int aptidx_match_topk(aptidx_ctx* ctx, int32_t cand, const float* S, int64_t nroi, int32_t topk, int32_t* best,
                      float* score, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if ((rc = check_ref(c, cand, true, false))) return rc;
    Reference& r = c->ref[cand];
    if (!S || !best || nroi <= 0) return set_error(c, APTIDX_E_INVALID_ARG, "match_topk: need S, best and nroi > 0");
    if (topk < 1 || topk > APTIDX_MAX_TOPK || topk > r.ng)
        return set_error(c, APTIDX_E_INVALID_ARG, "match_topk: topk = %d outside [1, min(ng = %lld, %d)]", topk,
                         (long long)r.ng, APTIDX_MAX_TOPK);
    static int max_optin = -1;
    if (max_optin < 0) cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (((size_t)c->nv + r.n_hat) * sizeof(float) > (size_t)max_optin)
        return set_error(c, APTIDX_E_INVALID_ARG, "match: %d directions do not fit one shared-memory signature row", c->nv);
    DevTmp tS, tb, ts;
    const float* dS;
    int32_t* db;
    float* ds;
    const size_t nout = (size_t)nroi * topk;
    if ((rc = dev_view(c, S, (size_t)nroi * c->nv, mem, tS, &dS))) return rc;
    if ((rc = dev_out(c, best, nout, mem, tb, &db))) return rc;
    if ((rc = dev_out(c, score, nout, mem, ts, &ds))) return rc;
    prof_begin(c, APTIDX_PHASE_MATCH);
    int launches = 0;
    if (topk == 1) {
        cudaError_t e = launch_match(c, &r, dS, nroi, db, ds);
        if (e != cudaSuccess) return cuda_check(c, e, "match");
        launches = 1;
    } else {
        // scores of a chunk of ROIs (at most 1 GiB), then a radix select per ROI
        const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nroi, ((int64_t)1 << 30) / (r.ng * 4)));
        const size_t need = (size_t)chunk * r.ng * sizeof(float);
        if (need > c->match_scratch_bytes) {
            free_ptr(c->d_match_scratch);
            c->match_scratch_bytes = 0;
            if ((rc = dev_alloc(c, (void**)&c->d_match_scratch, need))) return rc;
            c->match_scratch_bytes = need;
        }
        for (int64_t r0 = 0; r0 < nroi; r0 += chunk) {
            const int64_t n = std::min(chunk, nroi - r0);
            cudaError_t e = launch_match(c, &r, dS + r0 * c->nv, n, nullptr, nullptr, c->d_match_scratch);
            if (e == cudaSuccess)
                e = launch_topk(c, c->d_match_scratch, r.ng, n, topk, db + r0 * topk, ds ? ds + r0 * topk : nullptr);
            if (e != cudaSuccess) return cuda_check(c, e, "match_topk");
            launches += 2;
        }
    }
    prof_end(c, APTIDX_PHASE_MATCH, launches);
    if ((rc = copy_back(c, best, db, nout, mem))) return rc;
    if ((rc = copy_back(c, score, ds, nout, mem))) return rc;
    if (mem == APTIDX_MEM_HOST) return read_status(c);
    return APTIDX_OK;
}

int aptidx_match_phase(aptidx_ctx* ctx, int32_t n_cand, const int32_t* cand_off, const int32_t* ref,
                       const int32_t* sig, int32_t n_sig, const float* S, int64_t nroi, int32_t* phase, int32_t* best,
                       float* score, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if (n_cand < 1 || n_cand > kMaxCandidates || !cand_off || !ref || !sig || !S || nroi <= 0 || n_sig < 1)
        return set_error(c, APTIDX_E_INVALID_ARG, "match_phase: need 1 <= n_cand <= %d, offsets, slots, S, nroi > 0",
                         kMaxCandidates);
    if (!phase && !best && !score) return set_error(c, APTIDX_E_INVALID_ARG, "match_phase: no output");
    if (cand_off[0] != 0) return set_error(c, APTIDX_E_INVALID_ARG, "match_phase: cand_off[0] must be 0");
    for (int32_t k = 0; k < n_cand; ++k)
        if (cand_off[k + 1] <= cand_off[k] || cand_off[k + 1] > 64)
            return set_error(c, APTIDX_E_INVALID_ARG, "match_phase: candidate %d needs 1..64 channels", k);
    const int32_t n_ch = cand_off[n_cand];
    int64_t ng = -1;
    for (int32_t j = 0; j < n_ch; ++j) {
        if ((rc = check_ref(c, ref[j], true, false))) return rc;
        if (sig[j] < 0 || sig[j] >= n_sig)
            return set_error(c, APTIDX_E_INVALID_ARG, "match_phase: channel %d reads signature %d of %d", j, sig[j],
                             n_sig);
        if (ng >= 0 && c->ref[ref[j]].ng != ng)
            return set_error(c, APTIDX_E_INVALID_ARG, "match_phase: the look-up tables hold different orientation sets");
        if (!(c->ref[ref[j]].energy > 0.0))
            return set_error(c, APTIDX_E_INVALID_ARG, "match_phase: reference %d has no intensity at its strongest nodes",
                             ref[j]);
        ng = c->ref[ref[j]].ng;
    }
    static int max_optin = -1;
    if (max_optin < 0) cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    for (int32_t j = 0; j < n_ch; ++j)
        if (((size_t)c->nv + c->ref[ref[j]].n_hat) * sizeof(float) > (size_t)max_optin)
            return set_error(c, APTIDX_E_INVALID_ARG, "match_phase: %d directions do not fit one shared-memory row",
                             c->nv);
    DevTmp tS, tp, tb, ts, tn, tbw, tsw;
    const float* dS;
    int32_t *dp, *db, *dn;
    float* ds;
    const size_t nout = (size_t)n_cand * nroi;
    if ((rc = dev_view(c, S, (size_t)n_sig * nroi * c->nv, mem, tS, &dS))) return rc;
    if ((rc = dev_out(c, phase, (size_t)nroi, mem, tp, &dp))) return rc;
    if ((rc = dev_out(c, best, nout, mem, tb, &db))) return rc;
    if ((rc = dev_out(c, score, nout, mem, ts, &ds))) return rc;
    if (!db && (rc = dev_alloc(c, &tbw.p, nout * sizeof(int32_t)))) return rc;
    if (!db) db = static_cast<int32_t*>(tbw.p);
    if (!ds && (rc = dev_alloc(c, &tsw.p, nout * sizeof(float)))) return rc;
    if (!ds) ds = static_cast<float*>(tsw.p);
    std::vector<int32_t> nc((size_t)n_cand);
    for (int32_t k = 0; k < n_cand; ++k) nc[k] = cand_off[k + 1] - cand_off[k];
    if ((rc = dev_alloc(c, &tn.p, nc.size() * sizeof(int32_t)))) return rc;
    dn = static_cast<int32_t*>(tn.p);
    APTIDX_CUDA(c, cudaMemcpyAsync(dn, nc.data(), nc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    // channel sums of a chunk of ROIs (at most 1 GiB), then the argmin per ROI
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nroi, ((int64_t)1 << 30) / (ng * 4)));
    const size_t need = (size_t)chunk * ng * sizeof(float);
    if (need > c->match_scratch_bytes) {
        free_ptr(c->d_match_scratch);
        c->match_scratch_bytes = 0;
        if ((rc = dev_alloc(c, (void**)&c->d_match_scratch, need))) return rc;
        c->match_scratch_bytes = need;
    }
    prof_begin(c, APTIDX_PHASE_MATCH);
    int launches = 0;
    for (int32_t k = 0; k < n_cand; ++k) {
        for (int64_t r0 = 0; r0 < nroi; r0 += chunk) {
            const int64_t n = std::min(chunk, nroi - r0);
            cudaError_t e = cudaSuccess;
            for (int32_t j = cand_off[k]; j < cand_off[k + 1] && e == cudaSuccess; ++j) {
                e = launch_match(c, &c->ref[ref[j]], dS + ((int64_t)sig[j] * nroi + r0) * c->nv, n, nullptr, nullptr,
                                 c->d_match_scratch, j > cand_off[k], (float)(1.0 / c->ref[ref[j]].energy));
                ++launches;
            }
            if (e == cudaSuccess)
                e = launch_topk(c, c->d_match_scratch, ng, n, 1, db + (int64_t)k * nroi + r0, ds + (int64_t)k * nroi + r0);
            if (e != cudaSuccess) return cuda_check(c, e, "match_phase");
            ++launches;
        }
    }
    cudaError_t e = launch_phase(c, ds, dn, n_cand, nroi, dp);
    if (e != cudaSuccess) return cuda_check(c, e, "match_phase");
    prof_end(c, APTIDX_PHASE_MATCH, launches + 1);
    if ((rc = copy_back(c, phase, dp, (size_t)nroi, mem))) return rc;
    if ((rc = copy_back(c, best, db, nout, mem))) return rc;
    if ((rc = copy_back(c, score, ds, nout, mem))) return rc;
    APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));   // the temporaries are freed on return
    return read_status(c);
}

// Several signatures per ROI: signatures are grouped by type mask (one gather
// each) and their bands by up to APTIDX_MAX_BANDS per contraction; the ROI
// band of a pass spans the union of its bands, the kernels' epilogue takes
// each band's maximum and writes it to that signature's slab of S.
int aptidx_compute_signatures_multi(aptidx_ctx* ctx, int path, unsigned flags, int32_t n_sig,
                                    const uint32_t* type_mask, const int32_t* k_lo, const int32_t* k_hi, float* S,
                                    uint16_t* argk, int32_t* n_atoms, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if (c->nroi <= 0) return set_error(c, APTIDX_E_STATE, "compute_signatures_multi: set ROIs first");
    if (path != APTIDX_PATH_PLAIN_FP32 && path != APTIDX_PATH_TC_FP16)
        return set_error(c, APTIDX_E_INVALID_ARG, "unknown path %d", path);
    if (flags & ~APTIDX_NORMALISE_MAX) return set_error(c, APTIDX_E_INVALID_ARG, "unknown flags 0x%x", flags);
    c->use_pairs = true;
    if (n_sig < 1 || n_sig > 64 || !type_mask || !k_lo || !k_hi || !S)
        return set_error(c, APTIDX_E_INVALID_ARG, "compute_signatures_multi: need 1 <= n_sig <= 64, masks, bands, S");
    const int half = 1 << (c->m - 1);
    for (int s = 0; s < n_sig; ++s)
        if (k_lo[s] < 0 || k_hi[s] < k_lo[s] || k_hi[s] > half)
            return set_error(c, APTIDX_E_INVALID_ARG, "signature %d: band [%d, %d] outside [0, %d]", s, k_lo[s], k_hi[s],
                             half);
    const int64_t nS = c->nroi * (int64_t)c->nv;
    DevTmp tS, tA, tN;
    float* dS;
    uint16_t* dA;
    int32_t* dN;
    if ((rc = dev_out(c, S, (size_t)n_sig * nS, mem, tS, &dS))) return rc;
    if ((rc = dev_out(c, argk, (size_t)n_sig * nS, mem, tA, &dA))) return rc;
    if ((rc = dev_out(c, n_atoms, (size_t)n_sig * c->nroi, mem, tN, &dN))) return rc;

    // passes: signatures with the same type mask, in order of first use, in
    // groups of up to APTIDX_MAX_BANDS
    std::vector<std::vector<int>> passes;
    {
        std::vector<bool> used((size_t)n_sig, false);
        for (int s = 0; s < n_sig; ++s) {
            if (used[s]) continue;
            std::vector<int> grp;
            for (int t = s; t < n_sig; ++t)
                if (!used[t] && type_mask[t] == type_mask[s]) {
                    grp.push_back(t);
                    used[t] = true;
                }
            for (size_t i = 0; i < grp.size(); i += APTIDX_MAX_BANDS)
                passes.emplace_back(grp.begin() + i, grp.begin() + std::min(grp.size(), i + APTIDX_MAX_BANDS));
        }
    }
    // the gather buffer was sized for the context's type mask; a pass that
    // selects further atom types needs it sized for the union of the masks
    {
        uint32_t umask = 0;
        for (int s = 0; s < n_sig; ++s) umask |= type_mask[s];
        if (umask & ~c->type_mask) {
            const uint32_t m0 = c->type_mask;
            c->type_mask = umask;
            APTIDX_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
            cudaError_t e = launch_gather_count(c);
            c->type_mask = m0;
            if (e != cudaSuccess) return cuda_check(c, e, "ROI count");
            std::vector<int32_t> hnw((size_t)c->nroi);
            APTIDX_CUDA(c, cudaMemcpyAsync(hnw.data(), c->d_nw, (size_t)c->nroi * sizeof(int32_t),
                                           cudaMemcpyDeviceToHost, c->stream));
            APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
            int64_t total = 0;
            int32_t nwmax = 0;
            for (int64_t r = 0; r < c->nroi; ++r) {
                total += hnw[(size_t)r];
                nwmax = std::max(nwmax, hnw[(size_t)r]);
            }
            if (nwmax > APTIDX_MAX_ATOMS_PER_ROI) {
                APTIDX_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
                return set_error(c, APTIDX_E_OVERFLOW, "a ROI holds %d atoms of the requested types (limit %d)",
                                 nwmax, APTIDX_MAX_ATOMS_PER_ROI);
            }
            if (total > c->atoms_cap) {
                free_ptr(c->d_atoms);
                c->atoms_cap = 0;
                if ((rc = dev_alloc(c, (void**)&c->d_atoms, (size_t)total * sizeof(float4)))) return rc;
                c->atoms_cap = total;
            }
            if ((rc = read_status(c))) return rc;
        }
    }
    // the context's ROI bands and type mask are restored afterwards; cached
    // graphs may hold the B operand of other bands, so they are dropped
    clear_graphs(c);
    const uint32_t mask0 = c->type_mask;
    const std::vector<int32_t> band0 = c->h_band;
    const int32_t bmin0 = c->band_min, bmax0 = c->band_max;
    auto restore = [&]() {
        c->multi = BandSet();
        c->type_mask = mask0;
        c->h_band = band0;
        c->band_min = bmin0;
        c->band_max = bmax0;
        cudaMemcpyAsync(c->d_band, band0.data(), band0.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
        clear_graphs(c);
    };
    std::vector<int32_t> band((size_t)c->nroi * 2);
    for (const auto& ps : passes) {
        int lo_u = half, hi_u = 0;
        BandSet bs;
        bs.n = (int)ps.size();
        for (int b = 0; b < bs.n; ++b) {
            bs.lo[b] = k_lo[ps[b]];
            bs.hi[b] = k_hi[ps[b]];
            bs.off[b] = (int64_t)ps[b] * nS;
            lo_u = std::min(lo_u, bs.lo[b]);
            hi_u = std::max(hi_u, bs.hi[b]);
        }
        for (int64_t r = 0; r < c->nroi; ++r) {
            band[2 * r] = lo_u;
            band[2 * r + 1] = hi_u;
        }
        c->type_mask = type_mask[ps[0]];
        c->h_band = band;
        c->band_min = lo_u;
        c->band_max = hi_u;
        c->multi = bs;
        cudaError_t e = cudaMemcpyAsync(c->d_band, band.data(), band.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                        c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // the host band vector is reused
        if (e != cudaSuccess) {
            restore();
            return cuda_check(c, e, "band upload");
        }
        if (path == APTIDX_PATH_TC_FP16 && (rc = prepare_tc(c))) {
            restore();
            return rc;
        }
        if ((rc = launch_sequence(c, path, 0, dS, dA))) {
            restore();
            return rc;
        }
        if (dN)
            for (int b = 0; b < bs.n; ++b)
                cudaMemcpyAsync(dN + (int64_t)ps[b] * c->nroi, c->d_nw, (size_t)c->nroi * sizeof(int32_t),
                                cudaMemcpyDeviceToDevice, c->stream);
    }
    if (flags & APTIDX_NORMALISE_MAX) {
        prof_begin(c, APTIDX_PHASE_NORMALISE);
        cudaError_t e = launch_normalise(c, dS, (int64_t)n_sig * c->nroi);
        if (e != cudaSuccess) {
            restore();
            return cuda_check(c, e, "normalise");
        }
        prof_end(c, APTIDX_PHASE_NORMALISE, 1);
    }
    restore();
    if ((rc = copy_back(c, S, dS, (size_t)n_sig * nS, mem))) return rc;
    if ((rc = copy_back(c, argk, dA, (size_t)n_sig * nS, mem))) return rc;
    if ((rc = copy_back(c, n_atoms, dN, (size_t)n_sig * c->nroi, mem))) return rc;
    return read_status(c);
}

int aptidx_refine_roi_grid(aptidx_ctx* ctx, const float* S, int64_t nroi, float kappa, double spacing,
                           int32_t split, double* centres_out, int32_t* parent_out, int64_t cap, int64_t* n_out,
                           int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if (c->nroi <= 0) return set_error(c, APTIDX_E_STATE, "refine_roi_grid: set ROIs first");
    if (!S || !n_out || nroi != c->nroi)
        return set_error(c, APTIDX_E_INVALID_ARG, "refine_roi_grid: need S of the current %lld ROIs and n_out",
                         (long long)c->nroi);
    if (!(kappa > 0.f && kappa <= 1.f) || !(spacing > 0.0 && isfinite(spacing)) || split < 2 || split > 16 || cap < 0 ||
        (cap > 0 && !centres_out))
        return set_error(c, APTIDX_E_INVALID_ARG,
                         "refine_roi_grid: need 0 < kappa <= 1, spacing > 0, 2 <= split <= 16, cap >= 0 (and "
                         "centres_out when cap > 0)");
    DevTmp tS, tc, tp;
    const float* dS;
    double* dC;
    int32_t* dP;
    if ((rc = dev_view(c, S, (size_t)nroi * c->nv, mem, tS, &dS))) return rc;
    if ((rc = dev_out(c, centres_out, (size_t)cap * 3, mem, tc, &dC))) return rc;
    if ((rc = dev_out(c, parent_out, (size_t)cap, mem, tp, &dP))) return rc;
    int64_t nq = 0;
    cudaError_t e = launch_roi_refine(c, dS, kappa, spacing, split, cap > 0 ? dC : nullptr, dP, cap, &nq);
    if (e != cudaSuccess) return cuda_check(c, e, "ROI grid refinement");
    c->launches += cap > 0 ? 6 : 5;
    const int64_t n = nq * (int64_t)split * split * split;
    *n_out = n;
    const size_t nw = (size_t)std::min(n, cap);
    if ((rc = copy_back(c, centres_out, dC, nw * 3, mem))) return rc;
    if ((rc = copy_back(c, parent_out, dP, nw, mem))) return rc;
    APTIDX_CUDA(c, cudaStreamSynchronize(c->stream));
    return read_status(c);
}

int aptidx_compute_fsp(aptidx_ctx* ctx, int32_t grid_l, double k_max, float* amp, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if (c->nroi <= 0) return set_error(c, APTIDX_E_STATE, "compute_fsp: set ROIs first");
    if (!amp) return set_error(c, APTIDX_E_INVALID_ARG, "compute_fsp: need amp");
    if (grid_l < APTIDX_FSP_L_MIN || grid_l > APTIDX_FSP_L_MAX || grid_l % APTIDX_FSP_L_MIN != 0)
        return set_error(c, APTIDX_E_INVALID_ARG, "compute_fsp: grid_l = %d", grid_l);
    if (!(k_max > 0.0 && k_max <= 64.0)) return set_error(c, APTIDX_E_INVALID_ARG, "compute_fsp: k_max = %g", k_max);
    if (!tc_supported(c)) return set_error(c, APTIDX_E_INVALID_ARG, "compute_fsp: needs the sm_103 tensor cores");
    const int64_t L = grid_l;
    if (c->nroi * (L * L * L / 32768) >= ((int64_t)1 << 31))
        return set_error(c, APTIDX_E_INVALID_ARG, "compute_fsp: %lld ROIs at L = %d exceed 2^31 work items",
                         (long long)c->nroi, grid_l);
    const size_t n = (size_t)c->nroi * L * L * L;
    DevTmp t;
    float* d;
    if ((rc = dev_out(c, amp, n, mem, t, &d))) return rc;
    prof_begin(c, APTIDX_PHASE_GATHER);
    if ((rc = run_gather(c))) return rc;
    prof_end(c, APTIDX_PHASE_GATHER, 6);
    prof_begin(c, APTIDX_PHASE_SIGNATURE);
    cudaError_t e = launch_fsp_tc(c, grid_l, k_max, d);
    if (e != cudaSuccess) return cuda_check(c, e, "reciprocal-space signature");
    prof_end(c, APTIDX_PHASE_SIGNATURE, 1);
    if ((rc = copy_back(c, amp, d, n, mem))) return rc;
    return read_status(c);
}

int aptidx_refine_loss(aptidx_ctx* ctx, int32_t cand, const float* S, const double* q0, const double* omega,
                       int64_t nroi, float* loss, float* grad, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if ((rc = check_ref(c, cand, false, true))) return rc;
    if (!S || !q0 || !loss || nroi <= 0) return set_error(c, APTIDX_E_INVALID_ARG, "refine_loss: need S, q0, loss, nroi > 0");
    DevTmp tS, tq, tw, tl, tg;
    const float* dS;
    const double *dq, *dw = nullptr;
    float *dl, *dg;
    if ((rc = dev_view(c, S, (size_t)nroi * c->nv, mem, tS, &dS))) return rc;
    if ((rc = dev_view(c, q0, (size_t)nroi * 4, mem, tq, &dq))) return rc;
    if (omega && (rc = dev_view(c, omega, (size_t)nroi * 3, mem, tw, &dw))) return rc;
    if ((rc = dev_out(c, loss, (size_t)nroi, mem, tl, &dl))) return rc;
    if ((rc = dev_out(c, grad, (size_t)nroi * 3, mem, tg, &dg))) return rc;
    prof_begin(c, APTIDX_PHASE_REFINE);
    cudaError_t e = launch_refine_eval(c, &c->ref[cand], dS, dq, dw, nroi, dl, dg);
    if (e != cudaSuccess) return cuda_check(c, e, "refine loss");
    prof_end(c, APTIDX_PHASE_REFINE, 1);
    if ((rc = copy_back(c, loss, dl, (size_t)nroi, mem))) return rc;
    if ((rc = copy_back(c, grad, dg, (size_t)nroi * 3, mem))) return rc;
    if (mem == APTIDX_MEM_HOST) return read_status(c);
    return APTIDX_OK;
}

int aptidx_refine(aptidx_ctx* ctx, int32_t cand, const float* S, const double* q0, const int32_t* best, int64_t nroi,
                  int32_t iters, double* q_out, float* loss, int mem) {
    CTX_OR_FAIL(ctx);
    int rc;
    if ((rc = check_mem(c, mem))) return rc;
    if ((rc = check_ref(c, cand, best != nullptr, true))) return rc;
    if (!S || (!q0 && !best) || !q_out || nroi <= 0 || iters < 0 || iters > 1000)
        return set_error(c, APTIDX_E_INVALID_ARG, "refine: need S, q0 or best, q_out, nroi > 0, 0 <= iters <= 1000");
    DevTmp tS, tq, tb, to, tl;
    const float* dS;
    const double* dq = nullptr;
    const int32_t* db = nullptr;
    double* dqo;
    float* dl;
    if ((rc = dev_view(c, S, (size_t)nroi * c->nv, mem, tS, &dS))) return rc;
    if (best) {
        HostView<int32_t> hb;
        if ((rc = to_host(c, best, (size_t)nroi, mem, hb))) return rc;
        for (int64_t i = 0; i < nroi; ++i)
            if (hb[i] < 0 || hb[i] >= c->ref[cand].ng)
                return set_error(c, APTIDX_E_INVALID_ARG, "refine: best[%lld] = %d outside the table", (long long)i, hb[i]);
        if ((rc = dev_view(c, best, (size_t)nroi, mem, tb, &db))) return rc;
    } else if ((rc = dev_view(c, q0, (size_t)nroi * 4, mem, tq, &dq))) {
        return rc;
    }
    if ((rc = dev_out(c, q_out, (size_t)nroi * 4, mem, to, &dqo))) return rc;
    if ((rc = dev_out(c, loss, (size_t)nroi, mem, tl, &dl))) return rc;
    prof_begin(c, APTIDX_PHASE_REFINE);
    cudaError_t e = launch_refine_gn(c, &c->ref[cand], dS, dq, db, nroi, iters, dqo, dl);
    if (e != cudaSuccess) return cuda_check(c, e, "refine");
    prof_end(c, APTIDX_PHASE_REFINE, 1);
    if ((rc = copy_back(c, q_out, dqo, (size_t)nroi * 4, mem))) return rc;
    if ((rc = copy_back(c, loss, dl, (size_t)nroi, mem))) return rc;
    if (mem == APTIDX_MEM_HOST) return read_status(c);
    return APTIDX_OK;
}

}  // extern "C"
