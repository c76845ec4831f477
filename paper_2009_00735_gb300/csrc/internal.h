// internal.h -- context and launch prototypes of the aptidx library (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "aptidx.h"

namespace aptidx {

constexpr int kMaxCandidates = 8;
constexpr int kImgRows = 181;   // elevation -90..90 deg, 1 deg
constexpr int kImgCols = 360;   // azimuth 0..359 deg, 1 deg
constexpr int kTileDirs = 64;   // directions per signature work item

// device status word bits
constexpr int kStatusTimeout = 1;
constexpr int kStatusOverflow = 2;
constexpr int kStatusInvalid = 4;

// Bands whose maxima one signature pass takes (aptidx_compute_signatures_multi);
// n == 0: the ROI's own band only.  Band b is written at S + off[b] (elements).
struct BandSet {
    int n = 0;
    int lo[APTIDX_MAX_BANDS] = {0, 0, 0, 0};
    int hi[APTIDX_MAX_BANDS] = {0, 0, 0, 0};
    int64_t off[APTIDX_MAX_BANDS] = {0, 0, 0, 0};
};

struct Reference {
    float* d_node_sig = nullptr;   // [nv] normalised reference signature
    int32_t* d_top = nullptr;      // [n_hat] strongest nodes, strongest first
    float* d_top_val = nullptr;    // [n_hat] their values
    int32_t n_hat = 0;
    // reference image as bilinear cells, [180 x 360] or null: cell (i, j) holds
    // (I[i][j], I[i][j'], I[i+1][j], I[i+1][j']) with j' = (j + 1) mod 360
    float4* d_img4 = nullptr;
    void* d_lut = nullptr;         // [n_hat x ng_pad] (k-major), uint16 node indices when nv <= 65536, else int32
    int lut_bytes = 4;             // bytes per table entry (2 or 4)
    double* d_quats = nullptr;     // [ng x 4] test orientations of the table
    int64_t ng = 0;
    int64_t ng_pad = 0;            // row length of the table: ng rounded up to a multiple of 8
    int32_t nv_at_set = 0;
    double energy = 0.0;           // sum of the squared n_hat strongest values (Eq. 3 of an empty signature)
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    std::string err;

    // positions
    int64_t n_atoms = 0;
    float* d_pos = nullptr;        // [n x 3]
    uint8_t* d_types = nullptr;    // [n] or null
    int64_t pos_cap = 0;           // atoms d_pos holds room for (reused by a same-sized load)
    int64_t types_cap = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};

    // uniform cell grid over the positions
    double cell_h = 0.0;
    int dims[3] = {0, 0, 0};
    int64_t n_cells = 0;
    int64_t* d_cell_start = nullptr;   // [n_cells + 1]
    float4* d_cell_pos = nullptr;      // [n] positions in cell order, w = type (as float)

    // directions (padded to a multiple of kTileDirs with (1, 0, 0))
    int32_t nv = 0, nv_pad = 0;
    float4* d_dirs = nullptr;
    // the same directions in a spatially coherent order (Morton order of 1-degree
    // elevation-azimuth cells), w = the direction's index as int bits; the
    // refinement walks this order so that neighbouring lanes sample
    // neighbouring pixels of the reference image
    float4* d_dirs_sorted = nullptr;
    // antipodal pairs: one slot per pair (the lower index projected, its
    // partner written from it) and per unpaired direction, padded to whole
    // tiles; slot = (output direction, partner or -1).  Null without pairs.
    float4* d_slot_dirs = nullptr;
    int2* d_slot_idx = nullptr;
    int32_t nslot = 0, nslot_pad = 0, npairs = 0;
    bool use_pairs = true;           // cleared by APTIDX_DIRECT for one call
    float* d_gn_scratch = nullptr;   // one signature row per refinement CTA, in the order above
    size_t gn_scratch_bytes = 0;
    BandSet multi;                       // bands of the current pass (multi-signature calls)
    float* d_match_scratch = nullptr;   // Eq. 3 scores of a chunk of ROIs (top-k matching)
    size_t match_scratch_bytes = 0;

    // binning
    int m = 0;
    int32_t k_lo = 0, k_hi = 0;
    bool binning_set = false;
    float2* d_tw = nullptr;            // [2^m] (cos, sin)(2 pi j / 2^m), FP32
    int tw_m = 0;
    // tensor-core twiddle operand (B): [n_cols] hi/lo FP16 in canonical layout
    void* d_twb = nullptr;
    size_t twb_bytes = 0;
    int twb_key[3] = {-1, -1, -1};     // (m, band_min, groups)
    int tc_gb = 0;                     // frequency groups per B batch
    int tc_ng = 0;                     // groups in the global B operand
    uint32_t tc_tmem_cols = 0;
    bool tc_wide = false;              // some ROI band spans more groups than one B batch

    // ROIs
    int64_t nroi = 0;
    double* d_centres = nullptr;       // [nroi x 3]
    double* d_radii = nullptr;         // [nroi]
    float* d_scale = nullptr;          // [nroi] (float)((2^(m-1)-1)/R)
    int32_t* d_band = nullptr;         // [nroi x 2] (k_lo, k_hi)
    int32_t band_min = 0, band_max = 0;
    std::vector<int32_t> h_band;       // host copy of (k_lo, k_hi) per ROI
    uint32_t type_mask = 0xFFFFFFFFu;
    double r_max = 0.0;

    // gather output (CSR)
    int32_t* d_nw = nullptr;           // [nroi]
    int64_t* d_nw64 = nullptr;         // [nroi] widened counts (scan input)
    int64_t* d_off = nullptr;          // [nroi + 1]
    float4* d_atoms = nullptr;         // [total] centred FP32 (x, y, z, 0)
    int64_t atoms_cap = 0;
    int64_t atoms_total = 0;
    int32_t nw_max = 0;

    // scheduling scratch
    int32_t* d_order = nullptr;        // [nroi] ROI order (largest first)
    int32_t* d_counter = nullptr;      // [4] work counters
    int32_t* d_sort_hist = nullptr;    // [65536 + 1]
    int64_t* d_scan_tmp = nullptr;     // scan block sums
    size_t scan_tmp_elems = 0;

    // library-owned outputs used when the caller passes host buffers
    float* d_S = nullptr;
    uint16_t* d_argk = nullptr;
    int64_t S_cap = 0;

    // status word
    int* d_status = nullptr;

    // launch configuration (tiles per work item per path, MMA issuer warps),
    // set by the autotuner; rank_limit > 0 restricts a launch to the first
    // ranks of the ROI order (tuning runs)
    int tune_tpi[2] = {16, 16};
    int tune_iss = 4;
    int64_t rank_limit = 0;
    struct TuneCfg {
        int tpi, iss;
        float ms;
    };
    std::map<std::string, TuneCfg> tune_cache;
    bool tune_loaded = false;

    // CUDA graphs of compute_signatures calls, keyed by their arguments
    std::map<std::string, cudaGraphExec_t> graphs;
    // device blocks of the ROI set, the cell grid and its build released by a
    // reload, kept by exact size (at most kSpareBytes) for the next set of
    // equal sizes: a reload per step then allocates and frees nothing.  Every
    // reuse is ordered on `stream`, where the blocks were last used.
    std::vector<std::pair<void*, size_t>> spare;
    size_t spare_bytes = 0;
    cudaStream_t cap_stream = nullptr;

    Reference ref[kMaxCandidates];


    // profiling (CUDA events on the stream around phases)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    struct EvPair { int phase; cudaEvent_t a, b; };
    std::vector<EvPair> ev_pending;
    cudaEvent_t ev_open[APTIDX_N_PHASES] = {};
    double prof_ms[APTIDX_N_PHASES] = {};
    int64_t prof_calls[APTIDX_N_PHASES] = {};
    int64_t launches = 0;
};

// profiling helpers (no-ops unless profiling is enabled)
void prof_begin(Ctx* c, int phase);
void prof_end(Ctx* c, int phase, int kernels);

// error helpers ---------------------------------------------------------------
int set_error(Ctx* c, int code, const char* fmt, ...);
int cuda_check(Ctx* c, cudaError_t e, const char* what);
#define APTIDX_CUDA(ctx, call)                                    \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return ::aptidx::cuda_check(ctx, _e, #call); \
    } while (0)

int dev_alloc(Ctx* c, void** p, size_t bytes);
// hand a block from dev_alloc back for reuse by the same context (see Ctx::spare)
void dev_recycle(Ctx* c, void* p);
void release_spare(Ctx* c);
void dev_free(void* p);

// launches (all async on c->stream) -----------------------------------------
cudaError_t launch_bbox(const float* pos, int64_t n, float* d_minmax, cudaStream_t s);
cudaError_t launch_cell_build(Ctx* c, int32_t* d_cell_of, int32_t* d_k2, int32_t* d_idx, int32_t* d_v2,
                              int64_t* d_counts, int64_t* d_hist, int64_t* d_offs);
size_t cell_sort_hist_elems(int64_t n);
cudaError_t launch_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s);
size_t scan_tmp_elems(int64_t n);
cudaError_t launch_gather_count(Ctx* c);
cudaError_t launch_gather_fill(Ctx* c);
cudaError_t launch_roi_order(Ctx* c);
cudaError_t launch_roi_refine(Ctx* c, const float* S, float kappa, double spacing, int split, double* out,
                              int32_t* parent, int64_t cap, int64_t* n_qualified);
cudaError_t launch_twiddles(float2* tw, int m, cudaStream_t s);

// signature kernels
cudaError_t launch_signatures_plain(Ctx* c, float* S, uint16_t* argk, uint16_t* hist_out,
                                    int64_t hist_roi, int rank_mode);
cudaError_t launch_signatures_tc(Ctx* c, float* S, uint16_t* argk, uint16_t* hist_out,
                                 int64_t hist_roi);
int prepare_tc(Ctx* c);
bool tc_supported(Ctx* c);
cudaError_t launch_fsp_tc(Ctx* c, int L, double kmax, float* out);
bool tc_supported(Ctx* c);
cudaError_t launch_normalise(Ctx* c, float* S, int64_t rows = -1);   // rows of nv values; -1: nroi
size_t plain_smem_bytes(int m, int atom_cap);

// indexing / refinement
cudaError_t launch_top_nodes(Ctx* c, Reference* r);
cudaError_t launch_build_lut(Ctx* c, Reference* r, const double* d_quats, int64_t ng);
cudaError_t launch_match(Ctx* c, Reference* r, const float* S, int64_t nroi, int32_t* best, float* score,
                         float* scores_out = nullptr, bool accumulate = false, float weight = 1.0f);
cudaError_t launch_phase(Ctx* c, float* score, const int32_t* n_ch, int32_t n_cand, int64_t nroi, int32_t* phase);
cudaError_t launch_topk(Ctx* c, const float* scores, int64_t ng, int64_t nroi, int32_t topk, int32_t* best,
                        float* score);
cudaError_t launch_lut_export(Ctx* c, Reference* r, int32_t* out);
cudaError_t launch_refine_eval(Ctx* c, Reference* r, const float* S, const double* q0, const double* omega,
                               int64_t nroi, float* loss, float* grad);
cudaError_t launch_refine_gn(Ctx* c, Reference* r, const float* S, const double* q0, const int32_t* best,
                             int64_t nroi, int iters, double* q_out, float* loss);

}  // namespace aptidx

struct aptidx_ctx {
    aptidx::Ctx c;
};
