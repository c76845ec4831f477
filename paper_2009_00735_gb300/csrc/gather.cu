// gather.cu -- step (a1): ROI atom query and centring on the GPU.
//
// The paper queries the atoms of each ROI with a tree (supplement, cost term
// N_roi f R^3 rho log(V rho)).  Here the positions are bucketed once into a
// uniform cell grid (counting sort, cells ordered by atom index so results
// are deterministic), and one warp per ROI scans the cells that overlap the
// ROI's sphere.  Membership is the FP64 closed-ball test
// (dx*dx + dy*dy) + dz*dz <= R*R without fused multiply-add, and the centred
// coordinates x_i - p_c are rounded once to FP32 (Eq. 1: p_i - p_c).
#include <float.h>

#include "common.cuh"

namespace aptidx {

// -----------------------------------------------------------------------------
// bounding box
// -----------------------------------------------------------------------------
__device__ __forceinline__ int f2ord(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}

__global__ void k_bbox_init(int* mm) {
    if (threadIdx.x < 3) mm[threadIdx.x] = 0x7FFFFFFF;
    else if (threadIdx.x < 6) mm[threadIdx.x] = (int)0x80000000;
}

__global__ void k_bbox(const float* __restrict__ pos, int64_t n, int* mm) {
    int lo[3] = {0x7FFFFFFF, 0x7FFFFFFF, 0x7FFFFFFF};
    int hi[3] = {(int)0x80000000, (int)0x80000000, (int)0x80000000};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int o = f2ord(pos[3 * i + d]);
            lo[d] = min(lo[d], o);
            hi[d] = max(hi[d], o);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int d = 0; d < 3; ++d) {
            atomicMin(&mm[d], lo[d]);
            atomicMax(&mm[3 + d], hi[d]);
        }
    }
}

__global__ void k_bbox_decode(const int* mm, float* out) {
    int t = threadIdx.x;
    if (t < 6) {
        int i = mm[t];
        i = i >= 0 ? i : i ^ 0x7FFFFFFF;
        out[t] = __int_as_float(i);
    }
}

cudaError_t launch_bbox(const float* pos, int64_t n, float* d_minmax, cudaStream_t s) {
    int* mm = reinterpret_cast<int*>(d_minmax) + 6;   // caller provides 12 floats
    k_bbox_init<<<1, 32, 0, s>>>(mm);
    int blocks = (int)tmin<int64_t>((n + 255) / 256, 4096);
    k_bbox<<<blocks, 256, 0, s>>>(pos, n, mm);
    k_bbox_decode<<<1, 32, 0, s>>>(mm, d_minmax);
    return cudaGetLastError();
}

// -----------------------------------------------------------------------------
// exclusive scan of int64 (out[n] = total), up to 4096 * 4096 elements
// -----------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanBlock = kScanThreads * kScanPer;

size_t scan_tmp_elems(int64_t n) { return (size_t)((n + kScanBlock - 1) / kScanBlock) + 1; }

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* warp_sums, int64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        warp_sums[lane] = w;   // inclusive
    }
    __syncthreads();
    int64_t before = warp == 0 ? 0 : warp_sums[warp - 1];
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    return before + x - v;
}

__global__ void k_scan_blocks(const int64_t* __restrict__ in, int64_t* out, int64_t n, int64_t* sums) {
    __shared__ int64_t ws[32];
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    int64_t v[kScanPer];
    int64_t local = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        local += v[i];
    }
    int64_t ex = block_exclusive_scan(local, ws, &tot);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t* sums, int64_t nb) {
    __shared__ int64_t ws[32];
    __shared__ int64_t tot;
    int64_t base = threadIdx.x * kScanPer;
    int64_t v[kScanPer];
    int64_t local = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = base + i < nb ? sums[base + i] : 0;
        local += v[i];
    }
    int64_t ex = block_exclusive_scan(local, ws, &tot);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < nb) sums[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0) sums[nb] = tot;
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* sums, int64_t nb) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / kScanBlock];
    if (i == 0) out[n] = sums[nb];
}

cudaError_t launch_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s) {
    int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb > kScanBlock) return cudaErrorInvalidValue;
    if (nb == 0) {
        return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    }
    k_scan_blocks<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, tmp);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp, nb);
    k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, tmp, nb);
    return cudaGetLastError();
}

// -----------------------------------------------------------------------------
// cell grid
// -----------------------------------------------------------------------------
struct GridDesc {
    double lo[3];
    double inv_h;
    double h;
    int dims[3];
};

__device__ __forceinline__ int cell_coord(double x, double lo, double inv_h, int dim) {
    int i = (int)floor((x - lo) * inv_h);
    return min(max(i, 0), dim - 1);
}

__global__ void k_cell_of(const float* __restrict__ pos, int64_t n, GridDesc g, int32_t* cell_of,
                          unsigned long long* counts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int ix = cell_coord((double)pos[3 * i + 0], g.lo[0], g.inv_h, g.dims[0]);
        int iy = cell_coord((double)pos[3 * i + 1], g.lo[1], g.inv_h, g.dims[1]);
        int iz = cell_coord((double)pos[3 * i + 2], g.lo[2], g.inv_h, g.dims[2]);
        int c = ix + g.dims[0] * (iy + g.dims[1] * iz);
        cell_of[i] = c;
        atomicAdd(&counts[c], 1ull);
    }
}

// Atom indices in cell order, ascending inside every cell: a stable
// least-significant-digit radix sort of the cell ids (8 bits per pass) with
// the atom index as value, starting from ascending indices.  A pass splits the
// keys into tiles of kRsTile; k_rs_count counts each tile's digits,
// an exclusive scan of the counts (digit-major) gives every (digit, tile) its
// output offset, and k_rs_scatter writes each tile's keys in order: within a
// chunk of 256 keys a key's position is its digit's running offset plus the
// same-digit keys of lower lanes (warp match) and of lower warps.
constexpr int kRsThreads = 256;
constexpr int kRsChunks = 16;
constexpr int kRsTile = kRsThreads * kRsChunks;
constexpr int kRsWarps = kRsThreads / 32;

__global__ void __launch_bounds__(kRsThreads) k_rs_count(const int32_t* __restrict__ keys, int64_t n, int shift,
                                                         int64_t ntiles, int64_t* hist) {
    __shared__ int32_t h[256];
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
        const int64_t t0 = tile * kRsTile;
        for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
            const int64_t k = t0 + i;
            if (k < n) atomicAdd(&h[(keys[k] >> shift) & 255], 1);
        }
        __syncthreads();
        hist[(int64_t)threadIdx.x * ntiles + tile] = h[threadIdx.x];
        __syncthreads();
    }
}

// vin == nullptr: the values are the key positions (atom indices)
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const int32_t* __restrict__ kin,
                                                           const int32_t* __restrict__ vin, int64_t n, int shift,
                                                           int64_t ntiles, const int64_t* __restrict__ offs,
                                                           int32_t* kout, int32_t* vout) {
    __shared__ unsigned long long base[256];
    __shared__ int32_t wcnt[kRsWarps][257];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kRsWarps * 257; i += kRsThreads) (&wcnt[0][0])[i] = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        base[tid] = (unsigned long long)offs[(int64_t)tid * ntiles + tile];
        for (int ch = 0; ch < kRsChunks; ++ch) {
            const int64_t k = tile * kRsTile + (int64_t)ch * kRsThreads + tid;
            const bool valid = k < n;
            const int32_t key = valid ? kin[k] : 0;
            const int32_t val = valid ? (vin ? vin[k] : (int32_t)k) : 0;
            const int d = valid ? ((key >> shift) & 255) : 256;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const bool leader = lane == __ffs(peers) - 1;
            const int rank = __popc(peers & ((1u << lane) - 1u));
            if (leader) wcnt[warp][d] = __popc(peers);
            __syncthreads();
            if (valid) {
                long long pos = (long long)base[d] + rank;
                for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
                kout[pos] = key;
                vout[pos] = val;
            }
            __syncthreads();
            if (leader) {
                if (valid) atomicAdd(&base[d], (unsigned long long)__popc(peers));
                wcnt[warp][d] = 0;
            }
            __syncthreads();
        }
    }
}

__global__ void k_cell_fill(const float* __restrict__ pos, const uint8_t* __restrict__ types,
                            const int32_t* __restrict__ idx, int64_t n, float4* cell_pos) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = idx[k];
        float t = types ? (float)types[i] : 0.0f;
        cell_pos[k] = make_float4(pos[3 * (int64_t)i], pos[3 * (int64_t)i + 1], pos[3 * (int64_t)i + 2], t);
    }
}

static GridDesc grid_desc(const Ctx* c) {
    GridDesc g;
    for (int d = 0; d < 3; ++d) {
        g.lo[d] = c->lo[d];
        g.dims[d] = c->dims[d];
    }
    g.h = c->cell_h;
    g.inv_h = 1.0 / c->cell_h;
    return g;
}

// Build the cell grid of the loaded positions for the cell size c->cell_h.
// Scratch (caller-owned): cell_of, k2, idx, v2 [n] int32, counts [n_cells]
// int64, hist and offs [256 * ceil(n / kRsTile) + 1] int64.
size_t cell_sort_hist_elems(int64_t n) { return (size_t)256 * (size_t)((n + kRsTile - 1) / kRsTile) + 1; }

cudaError_t launch_cell_build(Ctx* c, int32_t* d_cell_of, int32_t* d_k2, int32_t* d_idx, int32_t* d_v2,
                              int64_t* d_counts, int64_t* d_hist, int64_t* d_offs) {
    cudaStream_t s = c->stream;
    GridDesc g = grid_desc(c);
    const int64_t n = c->n_atoms;
    int blocks = (int)tmin<int64_t>((n + 255) / 256, 8192);
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_counts, 0, sizeof(int64_t) * c->n_cells, s)) != cudaSuccess) return e;
    k_cell_of<<<blocks, 256, 0, s>>>(c->d_pos, n, g, d_cell_of, reinterpret_cast<unsigned long long*>(d_counts));
    if ((e = launch_scan_i64(d_counts, c->d_cell_start, c->n_cells, c->d_scan_tmp, s)) != cudaSuccess) return e;
    // radix passes over the bits of the largest cell id
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < c->n_cells) ++bits;
    const int passes = tmax(1, (bits + 7) / 8);
    const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
    const unsigned rblocks = (unsigned)tmin<int64_t>(tmax<int64_t>(ntiles, 1), (int64_t)c->sm_count * 8);
    const int32_t* kin = d_cell_of;
    const int32_t* vin = nullptr;
    int32_t* kbuf[2] = {d_k2, d_cell_of};
    int32_t* vbuf[2] = {d_idx, d_v2};
    for (int pass = 0; pass < passes && ntiles > 0; ++pass) {
        k_rs_count<<<rblocks, kRsThreads, 0, s>>>(kin, n, 8 * pass, ntiles, d_hist);
        if ((e = launch_scan_i64(d_hist, d_offs, 256 * ntiles, c->d_scan_tmp, s)) != cudaSuccess) return e;
        k_rs_scatter<<<rblocks, kRsThreads, 0, s>>>(kin, vin, n, 8 * pass, ntiles, d_offs, kbuf[pass & 1],
                                                    vbuf[pass & 1]);
        kin = kbuf[pass & 1];
        vin = vbuf[pass & 1];
    }
    k_cell_fill<<<blocks, 256, 0, s>>>(c->d_pos, c->d_types, vin, n, c->d_cell_pos);
    return cudaGetLastError();
}

// -----------------------------------------------------------------------------
// ROI gather: one warp per ROI, cells in fixed (z, y, x) order, atoms inside a
// cell in ascending index order, members compacted with a warp ballot.
// -----------------------------------------------------------------------------
struct GatherParams {
    GridDesc g;
    const int64_t* cell_start;
    const float4* cell_pos;
    const double* centres;
    const double* radii;
    int64_t nroi;
    uint32_t type_mask;
    int32_t* nw;           // count pass output
    const int64_t* off;    // fill pass input
    float4* atoms;         // fill pass output
    int64_t atoms_cap;     // entries of atoms (a fill past it records OVERFLOW and writes nothing)
    int* status;
};

template <bool kFill>
__global__ void __launch_bounds__(256) k_gather(GatherParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int64_t r = warp_global; r < p.nroi; r += nwarps) {
        const double cx = p.centres[3 * r], cy = p.centres[3 * r + 1], cz = p.centres[3 * r + 2];
        const double R = p.radii[r];
        const double R2 = __dmul_rn(R, R);
        int lo3[3], hi3[3];
        const double cc[3] = {cx, cy, cz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double a = (cc[d] - R - p.g.lo[d]) * p.g.inv_h - 1e-9;
            double b = (cc[d] + R - p.g.lo[d]) * p.g.inv_h + 1e-9;
            lo3[d] = (int)max(floor(a), 0.0);
            hi3[d] = (int)min(floor(b), (double)(p.g.dims[d] - 1));
        }
        int64_t count = 0;
        const int64_t base = kFill ? p.off[r] : 0;
        for (int iz = lo3[2]; iz <= hi3[2]; ++iz) {
            for (int iy = lo3[1]; iy <= hi3[1]; ++iy) {
                for (int ix = lo3[0]; ix <= hi3[0]; ++ix) {
                    // conservative cell-sphere distance test
                    const int ic[3] = {ix, iy, iz};
                    double d2 = 0.0;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        double clo = p.g.lo[d] + ic[d] * p.g.h;
                        double chi = clo + p.g.h;
                        double t = fmax(fmax(clo - cc[d], cc[d] - chi), 0.0);
                        d2 += t * t;
                    }
                    // edge cells absorb clamped atoms: do not skip them
                    bool edge = (ix == 0 || iy == 0 || iz == 0 || ix == p.g.dims[0] - 1 ||
                                 iy == p.g.dims[1] - 1 || iz == p.g.dims[2] - 1);
                    if (!edge && d2 > R2 * (1.0 + 1e-9) + 1e-12) continue;
                    const int64_t cell = ix + (int64_t)p.g.dims[0] * (iy + (int64_t)p.g.dims[1] * iz);
                    const int64_t s = p.cell_start[cell], e = p.cell_start[cell + 1];
                    for (int64_t j0 = s; j0 < e; j0 += 32) {
                        const int64_t j = j0 + lane;
                        bool in = false;
                        double dx = 0, dy = 0, dz = 0;
                        if (j < e) {
                            float4 a = p.cell_pos[j];
                            unsigned t = (unsigned)a.w;
                            bool sel = t < 32u && ((p.type_mask >> t) & 1u);
                            dx = __dsub_rn((double)a.x, cx);
                            dy = __dsub_rn((double)a.y, cy);
                            dz = __dsub_rn((double)a.z, cz);
                            double q = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                            in = sel && (q <= R2);
                        }
                        unsigned bal = __ballot_sync(0xffffffffu, in);
                        if (kFill && in) {
                            int64_t o = base + count + __popc(bal & lt_mask);
                            if (o < p.atoms_cap)
                                p.atoms[o] = make_float4(__double2float_rn(dx), __double2float_rn(dy),
                                                         __double2float_rn(dz), 0.0f);
                            else
                                raise_status(p.status, kStatusOverflow);
                        }
                        count += __popc(bal);
                    }
                }
            }
        }
        if (!kFill && lane == 0) {
            if (count > APTIDX_MAX_ATOMS_PER_ROI) raise_status(p.status, kStatusOverflow);
            p.nw[r] = (int32_t)tmin<int64_t>(count, 0x7FFFFFFF);
        }
    }
}

static GatherParams gather_params(Ctx* c) {
    GatherParams p;
    p.g = grid_desc(c);
    p.cell_start = c->d_cell_start;
    p.cell_pos = c->d_cell_pos;
    p.centres = c->d_centres;
    p.radii = c->d_radii;
    p.nroi = c->nroi;
    p.type_mask = c->type_mask;
    p.nw = c->d_nw;
    p.off = c->d_off;
    p.atoms = c->d_atoms;
    p.atoms_cap = c->d_atoms ? c->atoms_cap : 0;
    p.status = c->d_status;
    return p;
}

// counts N_w into d_nw
cudaError_t launch_gather_count(Ctx* c) {
    GatherParams p = gather_params(c);
    int blocks = (int)tmin<int64_t>((c->nroi * 32 + 255) / 256, (int64_t)c->sm_count * 16);
    k_gather<false><<<blocks, 256, 0, c->stream>>>(p);
    return cudaGetLastError();
}

__global__ void k_widen(const int32_t* __restrict__ nw, int64_t n, int64_t* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = nw[i];
}

// scans the counts into d_off, then writes the centred atoms
cudaError_t launch_gather_fill(Ctx* c) {
    k_widen<<<(unsigned)((c->nroi + 255) / 256), 256, 0, c->stream>>>(c->d_nw, c->nroi, c->d_nw64);
    cudaError_t e = launch_scan_i64(c->d_nw64, c->d_off, c->nroi, c->d_scan_tmp, c->stream);
    if (e != cudaSuccess) return e;
    GatherParams p = gather_params(c);
    int blocks = (int)tmin<int64_t>((c->nroi * 32 + 255) / 256, (int64_t)c->sm_count * 16);
    k_gather<true><<<blocks, 256, 0, c->stream>>>(p);
    return cudaGetLastError();
}

// -----------------------------------------------------------------------------
// ROI order for the persistent kernels: largest N_w first (longest processing
// time first), by a counting sort on 65535 - N_w.
// -----------------------------------------------------------------------------
__global__ void k_order_hist(const int32_t* __restrict__ nw, int64_t n, int32_t* hist, int32_t* n_big) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        atomicAdd(&hist[65535 - min(nw[i], 65535)], 1);
        if (nw[i] > kTcMaxAtoms) atomicAdd(n_big, 1);
    }
}

__global__ void __launch_bounds__(256) k_order_scan(int32_t* hist) {
    // single block of 256 threads, 256 consecutive entries each
    __shared__ int32_t part[256];
    const int t = threadIdx.x;
    int32_t* h = hist + t * 256;
    int32_t s = 0;
    for (int i = 0; i < 256; ++i) s += h[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        int32_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int32_t ex = part[t] - s;
    for (int i = 0; i < 256; ++i) {
        int32_t x = h[i];
        h[i] = ex;
        ex += x;
    }
}

__global__ void k_order_scatter(const int32_t* __restrict__ nw, int64_t n, int32_t* hist, int32_t* order) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        int pos = atomicAdd(&hist[65535 - min(nw[i], 65535)], 1);
        order[pos] = (int32_t)i;
    }
}

cudaError_t launch_roi_order(Ctx* c) {
    cudaStream_t s = c->stream;
    cudaError_t e = cudaMemsetAsync(c->d_sort_hist, 0, sizeof(int32_t) * 65536, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_counter + 1, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    unsigned b = (unsigned)((c->nroi + 255) / 256);
    k_order_hist<<<b, 256, 0, s>>>(c->d_nw, c->nroi, c->d_sort_hist, c->d_counter + 1);
    k_order_scan<<<1, 256, 0, s>>>(c->d_sort_hist);
    k_order_scatter<<<b, 256, 0, s>>>(c->d_nw, c->nroi, c->d_sort_hist, c->d_order);
    return cudaGetLastError();
}

// -----------------------------------------------------------------------------
// twiddle table (cos, sin)(2 pi j / 2^m) in FP32, from FP64 sincospi with the
// angle index reduced exactly in integers
// -----------------------------------------------------------------------------
__global__ void k_twiddles(float2* tw, int m) {
    int nb = 1 << m;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nb; j += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)j / (double)nb, &sn, &cs);
        tw[j] = make_float2((float)cs, (float)sn);
    }
}

cudaError_t launch_twiddles(float2* tw, int m, cudaStream_t s) {
    k_twiddles<<<((1 << m) + 255) / 256, 256, 0, s>>>(tw, m);
    return cudaGetLastError();
}

// -----------------------------------------------------------------------------
// local refinement of a cubic ROI grid (Section 3.4, aluminium bicrystal): a
// ROI qualifies when its peak signature value reaches kappa times the largest
// value over all ROIs; its grid cell is split into split^3 cells with a new
// ROI at every cell centre
// -----------------------------------------------------------------------------
namespace {

__global__ void __launch_bounds__(256) k_roi_peak(const float* __restrict__ S, int64_t nroi, int32_t nv, float* peak,
                                                  unsigned* gmax_bits) {
    __shared__ float red[8];
    for (int64_t r = blockIdx.x; r < nroi; r += gridDim.x) {
        const float* row = S + r * (int64_t)nv;
        float mx = 0.f;
        for (int v = threadIdx.x; v < nv; v += 256) mx = fmaxf(mx, row[v]);
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
            peak[r] = mx;
            atomicMax(gmax_bits, __float_as_uint(mx));   // non-negative floats order like their bits
        }
        __syncthreads();
    }
}

__global__ void k_roi_qualify(const float* __restrict__ peak, int64_t nroi, float kappa,
                              const unsigned* __restrict__ gmax_bits, int64_t* flag) {
    const float g = __uint_as_float(*gmax_bits);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nroi; r += (int64_t)gridDim.x * blockDim.x)
        flag[r] = (g > 0.f && peak[r] >= __fmul_rn(kappa, g)) ? 1 : 0;
}

// new ROI k = off[r] * split^3 + j, sub-cell j = ix + split (iy + split iz):
// centre = c + (i - (split - 1) / 2) * (spacing / split) per axis
__global__ void k_roi_split(const double* __restrict__ centres, const int64_t* __restrict__ flag,
                            const int64_t* __restrict__ off, int64_t nroi, double spacing, int split, double* out,
                            int32_t* parent, int64_t cap) {
    const int s3 = split * split * split;
    const double hh = __ddiv_rn(spacing, (double)split);
    const double mid = (double)(split - 1) * 0.5;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nroi * s3;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / s3;
        const int j = (int)(t % s3);
        if (!flag[r]) continue;
        const int64_t k = off[r] * s3 + j;
        if (k >= cap) continue;
        const int ix = j % split, iy = (j / split) % split, iz = j / (split * split);
        const int ii[3] = {ix, iy, iz};
        for (int d = 0; d < 3; ++d)
            out[3 * k + d] = __dadd_rn(centres[3 * r + d], __dmul_rn(__dadd_rn((double)ii[d], -mid), hh));
        if (parent) parent[k] = (int32_t)r;
    }
}

}  // namespace

cudaError_t launch_roi_refine(Ctx* c, const float* S, float kappa, double spacing, int split, double* out,
                              int32_t* parent, int64_t cap, int64_t* n_qualified) {
    const int64_t nroi = c->nroi;
    float* peak = nullptr;
    unsigned* gmax = nullptr;
    int64_t *flag = nullptr, *off = nullptr;
    cudaError_t e = cudaSuccess;
    if (dev_alloc(c, (void**)&peak, (size_t)nroi * sizeof(float)) ||
        dev_alloc(c, (void**)&gmax, sizeof(unsigned)) || dev_alloc(c, (void**)&flag, (size_t)nroi * sizeof(int64_t)) ||
        dev_alloc(c, (void**)&off, (size_t)(nroi + 1) * sizeof(int64_t)))
        e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaMemsetAsync(gmax, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) {
        k_roi_peak<<<(unsigned)tmin<int64_t>(nroi, (int64_t)c->sm_count * 16), 256, 0, c->stream>>>(S, nroi, c->nv,
                                                                                                     peak, gmax);
        k_roi_qualify<<<(unsigned)tmin<int64_t>((nroi + 255) / 256, 4096), 256, 0, c->stream>>>(peak, nroi, kappa,
                                                                                                gmax, flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_scan_i64(flag, off, nroi, c->d_scan_tmp, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n_qualified, off + nroi, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && cap > 0 && out) {
        const int64_t s3 = (int64_t)split * split * split;
        k_roi_split<<<(unsigned)tmin<int64_t>((nroi * s3 + 255) / 256, 65535), 256, 0, c->stream>>>(
            c->d_centres, flag, off, nroi, spacing, split, out, parent, cap);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(peak);
    dev_free(gmax);
    dev_free(flag);
    dev_free(off);
    return e;
}

}  // namespace aptidx
