/*
 * aptidx.h -- C ABI of the GB300 (sm_103a) library for real-space (RSP)
 * crystallographic signatures of atom probe data and their indexing, after
 * Kuehbach, Kasemer, Gault, Breen, "On Open and Strong-Scaling Tools for Atom
 * Probe Crystallography: High-Throughput Methods for Indexing Crystal
 * Structure and Orientation" (arXiv 2009.00735).
 *
 * The method (Section 2.2): for every region of interest (ROI) -- a sphere of
 * radius R around a point p_c -- project the ROI-centred atom positions onto
 * each direction of a geodesic sphere, bin the projected distances into a
 * 2^m-bin histogram (Eq. 1), take the histogram's Fourier amplitude spectrum,
 * and keep, per direction, the largest amplitude inside a band of frequency
 * bins.  The result is one spherical image (signature) per ROI, which is
 * matched against rotated reference signatures (Section 2.4, Eq. 3) and
 * refined to an orientation.
 *
 * Conventions
 *   - Every function returns an int status: APTIDX_OK (0) or an APTIDX_E_*
 *     code.  aptidx_last_error() gives a message for the last failure.
 *   - Pointers tagged `mem` are host memory (APTIDX_MEM_HOST) or device
 *     memory of the context's GPU (APTIDX_MEM_DEVICE).  The caller keeps
 *     ownership of every pointer it passes.  Inputs are copied into
 *     library-owned device memory before the call returns its work to the
 *     stream; outputs are written into caller-allocated buffers.
 *   - Work is queued on the context's CUDA stream.  Calls that return data
 *     to host memory synchronise that stream.  Calls that write device
 *     buffers do not: the caller orders later work on the same stream.
 *   - Device-side failures (a bounded wait that ran out, a count overflow)
 *     are recorded in a device status word and reported by the next
 *     synchronising call, or by aptidx_sync().
 *   - Layouts are row-major, C order.  Positions are FP32 nm, ROI centres
 *     and radii FP64 nm, directions FP32 unit vectors.
 *
 * Arithmetic contract (what the results equal)
 *   - Membership: atom i belongs to ROI c iff (dx*dx + dy*dy) + dz*dz <= R*R
 *     in FP64 with dx = (double)x_i - c_x (no fused multiply-add).  Centred
 *     coordinates are x_i - p_c rounded once to FP32.
 *   - Bin (Eq. 1 with dR = R / (2^(m-1) - 1), Fig. 2 caption):
 *       s = fma(u_z, x_z, fma(u_y, x_y, u_x * x_x))   (FP32, round-to-nearest)
 *       scale = (float)((2^(m-1) - 1) / R)
 *       b = clamp(2^(m-1) + floor(s * scale), 0, 2^m - 1)
 *     with s * scale the exact product.  Histograms are exact integers.
 *   - Spectrum: X(k) = sum_n h[n] exp(-2 pi i k n / 2^m), unnormalised,
 *     rectangular window; signature S(v) = max over the ROI's band of |X(k)|.
 */
#ifndef APTIDX_H
#define APTIDX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aptidx_ctx aptidx_ctx;

/* status codes */
#define APTIDX_OK              0
#define APTIDX_E_INVALID_ARG   1   /* a pointer, size or value is out of range */
#define APTIDX_E_CUDA          2   /* a CUDA runtime call failed */
#define APTIDX_E_OOM           3   /* device memory allocation failed */
#define APTIDX_E_TIMEOUT       4   /* a bounded device-side wait ran out */
#define APTIDX_E_OVERFLOW      5   /* a ROI or bin count exceeds what the path carries */
#define APTIDX_E_STATE         6   /* a required earlier call is missing */

/* memory spaces */
#define APTIDX_MEM_HOST        0
#define APTIDX_MEM_DEVICE      1

/* signature paths */
#define APTIDX_PATH_PLAIN_FP32 0   /* FP32 CUDA-core DFT of the histograms */
#define APTIDX_PATH_TC_FP16    1   /* histogram x DFT-matrix contraction on tcgen05 */

/* flags of aptidx_compute_signatures */
#define APTIDX_NORMALISE_MAX   1u  /* divide each ROI's signature by its largest value */
#define APTIDX_AUTOTUNE        2u  /* pick the launch configuration by timing candidates (once per shape) */
#define APTIDX_GRAPH           4u  /* capture the call's launches in a CUDA graph once, replay afterwards */
#define APTIDX_DIRECT          8u  /* project every direction, also those whose antipode is in the set */

/* limits */
#define APTIDX_MAX_ATOMS_PER_ROI 16777215   /* selected atoms per ROI (2^24 - 1) */
#define APTIDX_MIN_M 8
#define APTIDX_MAX_M 12                     /* Section 2.2: m in [8, 12] */

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t to queue all work on (NULL: the legacy default stream); the
 * caller keeps ownership of the stream.  On success *out receives the
 * context.  Errors: INVALID_ARG (out == NULL, bad device), CUDA. */
int aptidx_create(aptidx_ctx** out, int device, void* cuda_stream);

/* Synchronise the stream and free every library-owned buffer. */
int aptidx_destroy(aptidx_ctx* ctx);

/* Message of the last failing call on this context ("" if none).  The
 * string is owned by the context and valid until the next call. */
const char* aptidx_last_error(const aptidx_ctx* ctx);

/* Synchronise the context's stream and report the device status word:
 * TIMEOUT or OVERFLOW if a kernel recorded one since the last report.
 * Clears the word. */
int aptidx_sync(aptidx_ctx* ctx);

/* Library version (major * 10000 + minor * 100 + patch). */
int aptidx_version(void);

/* ---- inputs ------------------------------------------------------------- */

/* Atom positions of the reconstruction (Section 2.2: p_i).  xyz: n x 3 FP32
 * (x, y, z) in nm; types: n atom-type ids (NULL: all type 0).  Copies the
 * data and invalidates any previous ROI set; a set of the same n reuses the
 * device buffers.  Errors: INVALID_ARG (n <= 0, n >= 2^31, NULL xyz,
 * non-finite coordinate: the context then holds no positions), OOM, CUDA. */
int aptidx_load_positions(aptidx_ctx* ctx, const float* xyz, int64_t n, const uint8_t* types,
                          int mem);

/* Projection directions (Section 2.2: outer unit normals of the nodes of a
 * geodesic sphere, N_v = 40962 in the paper).  u: nv x 3 FP32 unit vectors
 * (|u| within 1e-5 of 1).  Directions whose exact negation is also in the set
 * (every node of a geodesic sphere has its antipode) are paired: the
 * signature paths project one direction of a pair and give the other the
 * same value and frequency bin, which is exact (the histogram along -u is the
 * mirror image of the one along u, with the same amplitude spectrum, unless
 * an atom's bin product is an exact integer; the kernels detect that case
 * and then project -u as well).  Errors: INVALID_ARG (nv <= 0, non-unit),
 * OOM, CUDA. */
int aptidx_set_directions(aptidx_ctx* ctx, const float* u, int32_t nv, int mem);

/* Histogram resolution 2^m bins (Eq. 1; APTIDX_MIN_M <= m <= APTIDX_MAX_M;
 * above 2^10 bins the kernels build each histogram in chunks of 1024 bins)
 * and the default signature band of frequency bins [k_lo, k_hi]
 * (supplement, Al bicrystal: the largest amplitude over a fixed band of bins),
 * 0 <= k_lo <= k_hi <= 2^(m-1).  flags: reserved, 0. */
int aptidx_set_binning(aptidx_ctx* ctx, int m, int32_t k_lo, int32_t k_hi, int flags);

/* The ROI list (Section 2.4: ROIs on a grid or randomly placed).
 * centres: nroi x 3 FP64 nm; radii: nroi FP64 nm in [1e-6, 1e6]; band_lo/band_hi:
 * per-ROI signature bands (NULL: the default band of aptidx_set_binning);
 * type_mask: bit t selects atoms of type t (0xFFFFFFFF: all).  All arrays
 * live in `mem`.  Requires positions, directions and binning.  Counts the
 * ROI atoms once to size the library's gather buffers.  Errors:
 * INVALID_ARG, STATE, OVERFLOW (a ROI holds more than
 * APTIDX_MAX_ATOMS_PER_ROI selected atoms), OOM, CUDA. */
int aptidx_set_rois(aptidx_ctx* ctx, const double* centres, const double* radii, int64_t nroi,
                    const int32_t* band_lo, const int32_t* band_hi, uint32_t type_mask, int mem);

/* Band of frequency bins holding the plane spacings [d_min, d_max] (nm) for a
 * ROI of radius R at 2^m bins (Fig. 2 caption: the sampling frequency is
 * f_s = 2^m / (2 (R + dR)) with dR = R / (2^(m-1) - 1), so frequency bin k
 * has the period W / k with W = 2 (R + dR); the supplement probes the
 * amplitude spectrum over the bin interval of a spacing interval):
 *   k_lo = ceil(W / d_max),  k_hi = floor(W / d_min)   (FP64).
 * Needs no context.  *k_lo and *k_hi (host) are written whenever the
 * arguments are valid.  Errors: INVALID_ARG (NULL outputs, 0 < d_min <=
 * d_max violated or not finite, R outside [1e-6, 1e6], m outside
 * [APTIDX_MIN_M, APTIDX_MAX_M], or a band that is empty or leaves
 * [0, 2^(m-1)], which aptidx_set_binning would refuse). */
int aptidx_band_for_spacing(double d_min, double d_max, double R, int m, int32_t* k_lo, int32_t* k_hi);

/* ---- the hot path -------------------------------------------------------- */

/* Signatures of every ROI: gather and centre the ROI atoms (FP64
 * membership), project them on every direction, histogram them (Eq. 1),
 * take the band of the amplitude spectrum and keep its maximum (Section
 * 2.2).  path: APTIDX_PATH_PLAIN_FP32 or APTIDX_PATH_TC_FP16.  flags: any of
 * APTIDX_NORMALISE_MAX; APTIDX_AUTOTUNE (the first call for a new shape --
 * bins, band width, mean ROI size, directions, device -- times candidate
 * launch configurations on the first 8 ROIs per SM and keeps the fastest;
 * with the environment variable APTIDX_TUNE_CACHE naming a file, choices
 * persist across processes); APTIDX_GRAPH (the launches of the call are
 * captured in a CUDA graph on first use for these output pointers and sizes
 * and replayed on later calls; input changes discard the graphs; the
 * profiler of aptidx_set_profiling then books the whole replay, gather and
 * ROI order included, as the signature phase);
 * APTIDX_DIRECT (no antipodal pairing: every direction is projected).
 * Outputs (in `mem`; NULL to skip): S nroi x nv FP32; argk nroi x nv u16 (the
 * lowest frequency bin attaining the maximum; not written when normalising
 * is the only change); n_atoms nroi int32 (N_w per ROI).
 * With mem == APTIDX_MEM_HOST the call copies the results back and
 * synchronises.  Errors: STATE, INVALID_ARG, OVERFLOW, TIMEOUT, OOM, CUDA. */
int aptidx_compute_signatures(aptidx_ctx* ctx, int path, unsigned flags, float* S, uint16_t* argk,
                              int32_t* n_atoms, int mem);

/* Several signatures per ROI in one call (Section 3.1: signatures per atom
 * type and per lattice-plane family distinguish crystal structures; the
 * aluminium bicrystal uses {002}, {220} and {111} signatures).  Signature s
 * uses the ROI atoms whose type bit is set in type_mask[s] and the
 * frequency band [k_lo[s], k_hi[s]] (the same band for every ROI).
 * Signatures with the same type mask share one gather and one spectrum
 * contraction over the union of their bands, up to APTIDX_MAX_BANDS bands
 * per contraction, the band maxima taken in the kernels' epilogue.
 * type_mask, k_lo, k_hi: host arrays of n_sig (1 <= n_sig <= 64).
 * S: n_sig x nroi x nv FP32 (signature-major); argk: same shape uint16
 * (NULL to skip); n_atoms: n_sig x nroi int32 (NULL to skip); these three
 * in `mem`.
 * flags: APTIDX_NORMALISE_MAX or 0.  The context's ROI bands and type mask
 * are left as they were; masks that select atom types beyond the context's
 * mask grow the gather buffer to the union of the masks.  Errors:
 * INVALID_ARG, STATE, OOM, CUDA, TIMEOUT, OVERFLOW (a ROI above
 * APTIDX_MAX_ATOMS_PER_ROI atoms of the requested types). */
#define APTIDX_MAX_BANDS 4
int aptidx_compute_signatures_multi(aptidx_ctx* ctx, int path, unsigned flags, int32_t n_sig,
                                    const uint32_t* type_mask, const int32_t* k_lo, const int32_t* k_hi, float* S,
                                    uint16_t* argk, int32_t* n_atoms, int mem);

/* Debug/parity: the 2^m-bin histograms of ROI `roi` for every direction, as
 * computed by the histogram stage of `path` (same kernel code).  h: nv x 2^m
 * u16 in `mem`. */
int aptidx_get_histograms(aptidx_ctx* ctx, int64_t roi, int path, uint16_t* h, int mem);

/* Debug/parity: the centred FP32 coordinates of ROI `roi` in gather order.
 * xc: cap x 3 FP32 in `mem`; *n_out receives N_w (written even if cap is
 * too small, in which case nothing is copied and OVERFLOW is returned). */
int aptidx_get_roi_atoms(aptidx_ctx* ctx, int64_t roi, float* xc, int64_t cap, int64_t* n_out,
                         int mem);

/* Local octree-like refinement of a cubic ROI grid (Section 3.4, aluminium
 * bicrystal): a ROI of the current set qualifies when the maximum of its
 * signature row reaches kappa times the largest signature value over all
 * ROIs (the paper's "kappa >= 0.75 normalised image intensity", read with
 * the dataset's largest value as the normalisation); the cubic grid cell of
 * edge `spacing` centred on each qualifying ROI is split into split^3 cells
 * and a new ROI is placed at every cell centre: new ROI k = q * split^3 + j
 * for the q-th qualifying ROI (in ROI order) and cell j = ix + split * (iy +
 * split * iz), centre + (i - (split - 1) / 2) * spacing / split per axis in
 * FP64.  S: nroi x nv FP32 signatures of the current ROIs (raw, or
 * normalised the same way for every ROI) in `mem`; nroi must equal the
 * context's ROI count.  centres_out: cap x 3 FP64, parent_out: cap int32
 * (the coarse ROI, NULL to skip), both in `mem`; *n_out (host) receives the
 * number of new ROIs, which may exceed cap (then the first cap are
 * written).  0 < kappa <= 1, spacing > 0, 2 <= split <= 16.  The new ROIs
 * are not installed: pass them to aptidx_set_rois for the second pass.
 * Errors: INVALID_ARG, STATE, OOM, CUDA. */
int aptidx_refine_roi_grid(aptidx_ctx* ctx, const float* S, int64_t nroi, float kappa, double spacing,
                           int32_t split, double* centres_out, int32_t* parent_out, int64_t cap, int64_t* n_out,
                           int mem);

/* Reciprocal-space signature (Eq. 2, the FSP method of Section 2.2 after
 * Vurpillot et al.): for every ROI of the current set (and type mask),
 * |F(k)| with F(k) = sum_w exp(-2 pi i k . (p_w - p_c)) over the ROI's
 * atoms (centred FP32 coordinates of the gather, nm), on the cubic grid
 * k = (k_x, k_y, k_z), k_a = -k_max + i_a dk, i_a < L, dk = 2 k_max / (L - 1),
 * k in nm^-1 (the supplement's grid over [-2 pi, 2 pi]^3 gives k_max = 2 pi;
 * its benchmarks use L = 64 and L = 512).  grid_l = L: a multiple of 64 in
 * [APTIDX_FSP_L_MIN, APTIDX_FSP_L_MAX].  amp: nroi x L x L x L FP32,
 * amp[((roi * L + ix) * L + iy) * L + iz], in `mem` (L = 512 is 512 MiB per
 * ROI: pass ROI sets that fit).  Computed as tensor-core GEMMs with fp16
 * operands and FP32 accumulation (sm_103 only).  0 < k_max <= 64.
 * Errors: INVALID_ARG (no tensor cores, bad grid_l or k_max, more than 2^31
 * work items), STATE, OOM, CUDA, TIMEOUT. */
#define APTIDX_FSP_L_MIN 64
#define APTIDX_FSP_L_MAX 512
int aptidx_compute_fsp(aptidx_ctx* ctx, int32_t grid_l, double k_max, float* amp, int mem);

/* ---- indexing (supplement "Indexing algorithm", Eq. 3) ---------------------- */

/* Reference of crystal-structure candidate `cand` (0 <= cand < 8):
 * node_sig: nv FP32 normalised reference signature on the current
 * directions (its n_hat strongest nodes enter Eq. 3);
 * img: 181 x 360 FP32 elevation-azimuth image of the same reference
 * (row i: elevation -90 + i degrees; column j: azimuth j degrees), used by
 * refinement; may be NULL if refinement is not used.
 * 1 <= n_hat <= nv.  Errors: INVALID_ARG, STATE, OOM, CUDA. */
int aptidx_set_reference(aptidx_ctx* ctx, int32_t cand, const float* node_sig, int32_t n_hat,
                         const float* img, int mem);

/* Look-up table of candidate `cand` for test orientations quats (ng x 4
 * FP64 unit quaternions (w, x, y, z), mapping crystal to lab): entry
 * (g, k) = the direction index nearest to R(q_g) n_k for the k-th strongest
 * reference node n_k.  Errors: INVALID_ARG, STATE, OOM, CUDA. */
int aptidx_build_lut(aptidx_ctx* ctx, int32_t cand, const double* quats, int64_t ng, int mem);

/* Debug/parity: the look-up table of candidate `cand`, lut[g * n_hat + k]
 * (ng x n_hat int32 in `mem`); *n_hat_out receives n_hat (may be NULL). */
int aptidx_get_lut(aptidx_ctx* ctx, int32_t cand, int32_t* lut, int32_t* n_hat_out, int mem);

/* Eq. 3 for every ROI: Delta(g) = sum_k (S[roi, lut[g, k]] - ref[n_k])^2
 * over the candidate's look-up table; best[roi] = argmin_g (ties: lowest
 * g), score[roi] = Delta(best).  S: nroi x nv FP32 normalised signatures in
 * `mem`; best: nroi int32; score: nroi FP32 (NULL to skip).  Errors:
 * INVALID_ARG, STATE, OOM, CUDA. */
int aptidx_match(aptidx_ctx* ctx, int32_t cand, const float* S, int64_t nroi, int32_t* best,
                 float* score, int mem);

/* Eq. 3 keeping the topk best orientations per ROI (the paper keeps up to
 * 1000 solutions per ROI, supplement "Indexing algorithm"):
 * best[roi * topk + i] and score[roi * topk + i], i < topk, ascending by
 * (Delta, g) -- ties resolve to the lower g, so topk = 1 equals
 * aptidx_match.  1 <= topk <= min(ng, APTIDX_MAX_TOPK).  Delta is
 * accumulated in FP32 in k order as in aptidx_match.  The scores of a chunk
 * of ROIs are staged on the device (at most 1 GiB, library-owned) and
 * reduced by a radix select per ROI.  S, best, score (NULL to skip) in
 * `mem`.  Errors: INVALID_ARG, STATE, OOM, CUDA. */
#define APTIDX_MAX_TOPK 1024
int aptidx_match_topk(aptidx_ctx* ctx, int32_t cand, const float* S, int64_t nroi, int32_t topk, int32_t* best,
                      float* score, int mem);

/* Phase and orientation from several signatures per candidate (Section 2.3,
 * "Indexing": every ROI's signatures are compared with the rotated references
 * of every crystal-structure candidate; the supplement's Al-Li-Mg-Ag case
 * compares three reference patterns, one for pure Al and one for each
 * sub-lattice of Al3Li, each probed in its own plane-spacing band).
 * Candidate c owns the signature channels j in [cand_off[c], cand_off[c+1]);
 * channel j compares the measured signatures S[sig[j]] (S: n_sig x nroi x nv
 * FP32, normalised, the layout of aptidx_compute_signatures_multi) with the
 * reference of slot ref[j] (aptidx_set_reference; its look-up table built by
 * aptidx_build_lut on one orientation set shared by every slot used).
 *   Delta_c(g) = (1 / n_c) sum_j Delta_ref[j](g) / E_ref[j],  n_c = cand_off[c+1] - cand_off[c],
 * with Delta of Eq. 3 accumulated in FP32 (channels in j order) and E the
 * reference's energy, the sum of its n_hat strongest values squared (FP64,
 * at aptidx_set_reference): Eq. 3 of an empty signature.  The paper leaves
 * open how image differences compare across candidates; relative to E a
 * channel scores 0 for a perfect match and 1 for no signal, whatever the
 * number of its reference's peaks.  A reference with E = 0 is refused.
 * best[c * nroi + roi] = argmin_g Delta_c(g) (ties: lowest g);
 * score[c * nroi + roi] = Delta_c(best); phase[roi] = the candidate with the
 * lowest score (ties: lowest c).  cand_off, ref, sig: host arrays
 * (1 <= n_cand <= 8, every candidate at least one channel); S, phase, best,
 * score (each output may be NULL) in `mem`.  Scores of a chunk of ROIs are
 * staged on the device (at most 1 GiB, library-owned).  Errors: INVALID_ARG,
 * STATE, OOM, CUDA. */
int aptidx_match_phase(aptidx_ctx* ctx, int32_t n_cand, const int32_t* cand_off, const int32_t* ref,
                       const int32_t* sig, int32_t n_sig, const float* S, int64_t nroi, int32_t* phase, int32_t* best,
                       float* score, int mem);

/* ---- orientation refinement ------------------------------------------------ */

/* Loss and gradient of the misfit between measured signatures and the
 * candidate's reference image sampled bilinearly at R^T u:
 *   L_roi = sum_v (S[roi, v] - I(alpha, beta of R^T u_v))^2,
 * leaving out directions whose crystal-frame elevation exceeds 89 degrees
 * in magnitude.  The rotation is R = exp([omega]x) R(q0) (q0: nroi x 4 FP64
 * unit quaternions; omega: nroi x 3 FP64 axis-angle vectors, or NULL for
 * omega = 0).  loss: nroi FP32 (the forward kernel).  grad (NULL to skip):
 * nroi x 3 FP32 dL/domega (the backward kernel; with omega = NULL this is
 * the derivative with respect to a lab-frame rotation exp([delta]x) R(q0) at
 * delta = 0).  All arrays in `mem`.  Errors: STATE (no reference image),
 * INVALID_ARG, OOM, CUDA. */
int aptidx_refine_loss(aptidx_ctx* ctx, int32_t cand, const float* S, const double* q0, const double* omega,
                       int64_t nroi, float* loss, float* grad, int mem);

/* `iters` Gauss-Newton steps per ROI: delta = -(J^T J + lambda I)^-1 J^T r
 * with lambda = 1e-6 tr(J^T J), R <- exp([delta]x) R, FP64 renormalisation.
 * The start is q0[roi] (nroi x 4 FP64), or, when `best` (nroi int32) is
 * given, the candidate's test orientation best[roi] from the last
 * aptidx_build_lut (as aptidx_match returns it); q0 may then be NULL.
 * q_out: nroi x 4 FP64 (w >= 0); loss: nroi FP32 at q_out (NULL to skip).
 * All arrays in `mem`.  Errors: STATE, INVALID_ARG, OOM, CUDA. */
int aptidx_refine(aptidx_ctx* ctx, int32_t cand, const float* S, const double* q0, const int32_t* best,
                  int64_t nroi, int32_t iters, double* q_out, float* loss, int mem);

/* ---- capabilities and profiling ------------------------------------------- */

/* The launch configuration the next call on `path` uses: 64-direction tiles
 * per work item and, on the tensor-core path, MMA issuer warps (else 0). */
int aptidx_get_tuning(aptidx_ctx* ctx, int path, int32_t* tiles_per_item, int32_t* issuers);

/* 1 if `path` can run on the context's device, else 0. */
int aptidx_path_supported(aptidx_ctx* ctx, int path);

/* Phases timed when profiling is on. */
#define APTIDX_PHASE_GATHER    0   /* ROI count, offsets, gather + centring (a1) */
#define APTIDX_PHASE_ORDER     1   /* longest-first ROI order */
#define APTIDX_PHASE_SIGNATURE 2   /* projection, histogram, spectrum, band max (a2-a5) */
#define APTIDX_PHASE_NORMALISE 3
#define APTIDX_PHASE_MATCH     4   /* Eq. 3 (a6) */
#define APTIDX_PHASE_REFINE    5   /* Gauss-Newton (a7) */
#define APTIDX_N_PHASES        6

/* enable != 0: record CUDA events on the context's stream around every
 * phase of the following calls and count the kernels they launch; resets
 * the totals.  enable == 0: stop recording. */
int aptidx_set_profiling(aptidx_ctx* ctx, int enable);

/* Synchronise and return the totals since profiling was enabled:
 * phase_ms[APTIDX_N_PHASES] summed CUDA-event milliseconds, phase_calls
 * [APTIDX_N_PHASES] how many times each phase ran, *launches the number of
 * library kernels launched.  Any pointer may be NULL. */
int aptidx_get_profile(aptidx_ctx* ctx, double* phase_ms, int64_t* phase_calls, int64_t* launches);

/* Read bandwidth of this device's L2 cache, the roof of the gather-bound
 * kernels (Eq. 3's look-up table reads, the refinement's image taps): a
 * kernel reads a `bytes`-sized device buffer (small enough to stay in L2;
 * 1 MiB .. 96 MiB, a multiple of 16) `iters` times with 16-byte loads that
 * bypass L1, after one untimed pass; *gbs = bytes x iters / kernel time (CUDA
 * events on the context's stream).  Allocates and frees the buffer; a
 * measurement helper, not a step of the method.  Errors: INVALID_ARG, OOM,
 * CUDA. */
int aptidx_probe_l2(aptidx_ctx* ctx, int64_t bytes, int32_t iters, double* gbs);

/* Throughput of shared-memory atomic adds on this device, the roof of the
 * histogram of Eq. 1 as the signature kernels build it (one 32-bit
 * red.shared.add per warp lane, each lane in its own bank, rows drawn at
 * random): one block of `threads` threads (a multiple of 32 in [32, 1024])
 * per SM, each thread issuing `iters` x 16 increments into a 128 KB shared
 * array, after one untimed pass.  *incr_per_s = lane increments per second
 * over the whole device (CUDA events on the context's stream);
 * *reds_per_sm_cycle (may be NULL) = 32-lane atomic instructions per SM and
 * SM clock cycle (clock64 inside the blocks).  Each block checks that its
 * array holds every increment (else APTIDX_E_CUDA).  A measurement helper, not
 * a step of the method.  Errors: INVALID_ARG, OOM, CUDA. */
int aptidx_probe_smem_atomics(aptidx_ctx* ctx, int32_t threads, int32_t iters, double* incr_per_s,
                              double* reds_per_sm_cycle);

/* ---- no-allocation variant ------------------------------------------------ */

/* The paper has no counterpart of this call; it serves callers that cannot
 * allocate device memory: code that runs while a CUDA graph is being
 * captured, a host framework that owns every device allocation through its
 * own pool, or a plugin that may not call cudaMalloc from its callback.
 * It computes the FP32 signatures of aptidx_compute_signatures
 * (APTIDX_PATH_PLAIN_FP32, no normalisation) for ROIs whose atoms the caller
 * has already gathered and centred, and needs no context.
 *
 *   xc4     device, 16-byte aligned: centred atom coordinates as rows of four
 *           floats (x, y, z, unused); ROI r owns rows [off[r], off[r+1])
 *   off     device, nroi + 1 int64 row offsets
 *   radii   device, nroi FP64 ROI radii in [1e-6, 1e6] nm
 *   u       device, nv x 3 FP32 unit directions (|u| within 1e-5 of 1)
 *   m, k_lo, k_hi: 2^m bins and the signature band, as in aptidx_set_binning
 *   S       device output, nroi x nv FP32
 *   status  device int or NULL: the kernels OR APTIDX_STATUS_* bits into it
 *           (OVERFLOW: a ROI above APTIDX_MAX_ATOMS_PER_ROI atoms; INVALID: a
 *           radius outside [1e-6, 1e6] or NaN, or a direction that is not a
 *           unit vector; TIMEOUT: a bounded wait that ran out).  A ROI flagged
 *           OVERFLOW or for its radius gets a zero row of S.  The caller
 *           clears the word.
 *   cuda_stream  the stream to queue on (NULL: the legacy default stream)
 *
 * Work is queued on the stream and the call returns without waiting.  It
 * allocates nothing: what the call derives from its inputs lives in one
 * library-owned scratch array of APTIDX_NOALLOC_SCRATCH_BYTES (2.5 MiB) that
 * every GPU loading the library holds until the process exits.  Hence
 * nroi <= APTIDX_NOALLOC_MAX_ROIS and nv <= APTIDX_NOALLOC_MAX_DIRS; larger
 * sizes, m outside [APTIDX_MIN_M, APTIDX_MAX_M], a bad band or a misaligned
 * xc4 return APTIDX_E_INVALID_ARG before any work is queued.  Every call
 * shares the scratch array, which keeps the last call's contents: calls
 * whose work overlaps on the GPU (other streams, other threads) race, so
 * order them on one stream.  The first call on a device looks up the
 * array's device address (once per device, with that device current) and
 * keeps it for the life of the process; make that first call before any
 * stream capture.  The kept address does not survive cudaDeviceReset: after
 * a reset of a device, this call must not be used on it again in the same
 * process.
 * Returns APTIDX_OK, APTIDX_E_INVALID_ARG or APTIDX_E_CUDA. */
#define APTIDX_NOALLOC_MAX_ROIS 65536
#define APTIDX_NOALLOC_MAX_DIRS 65536
#define APTIDX_NOALLOC_SCRATCH_BYTES (2621440)
#define APTIDX_STATUS_TIMEOUT  1
#define APTIDX_STATUS_OVERFLOW 2
#define APTIDX_STATUS_INVALID  4
int aptidx_signatures_noalloc(const float* xc4, const int64_t* off, const double* radii, int64_t nroi,
                              const float* u, int32_t nv, int m, int32_t k_lo, int32_t k_hi, float* S,
                              int* status, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* APTIDX_H */
