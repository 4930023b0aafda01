/*
 * epic_interp — EpicFlow's sparse-to-dense interpolator on one GB300 GPU.
 *
 * Given an edge-cost map C and a sparse match set M = {(p_m, p'_m)}, the
 * library produces the dense flow field of Algorithm 1 (LA form) of Revaud et
 * al., "EpicFlow: Edge-Preserving Interpolation of Correspondences for Optical
 * Flow" (arXiv:1501.02565):
 *   (a) the geodesic assignment map L(p) = argmin_m D_G(p, p_m) and the
 *       distance D(p) = D_G(p, L(p))     (Sec. 3.4 "Geodesic Voronoi diagram";
 *       D_G of Eq. 3 on the 8-connected pixel grid, step p->q costing
 *       |p-q| (C(p)+C(q))/2);
 *   (b) the match graph G joining matches whose cells touch, weighted by the
 *       geodesic distance restricted to the two cells (Sec. 3.4);
 *   (c) for every match, its K nearest matches on G (Algorithm 1, step 5, the
 *       approximation D~ of Eq. 4) and a locally-weighted affine fit with
 *       kernel exp(-a D) (Eq. 1-2, restricted to N_K as in Sec. 3.2);
 *   (d) the dense write-out F(p) = A_{L(p)} p + t_{L(p)} (Algorithm 1, steps
 *       7-8, LA form), returned as flow F(p) - p.
 * Options: the Nadaraya-Watson estimator of Eq. 1 in place of the LA fit
 * (the flow is then constant over each cell, Algorithm 1), and the
 * consistency pruning of Sec. 4.1 ("Pruning of matches") before the
 * interpolation.
 *
 * Conventions shared by every entry point
 *   - Images are row-major, x = column, y = row; pixel centres are integer.
 *   - cost_map: float32 [H*W], every value finite and >= 0 (edge
 *     strengths).  The relaxation adds exact fixed-point step costs.  With
 *     the default warp-tile relaxation each pair gets its own unit,
 *     2^-(31 - s): s = 0 (units of 2^-31) unless the pair's largest cost
 *     reaches 2 or a bound on its distances (its largest cost times the
 *     distance from any pixel to a seed, counted in relaxation tiles)
 *     reaches 1024, then the smallest s that holds both; costs up to 2^21
 *     and distances up to 2^30 fit.  The exact variant, the no-allocation
 *     entry point and the relaxation schedules 0 and 1 keep the unit 2^-31:
 *     costs below 2, distances below 1024.  A value outside the range, or a
 *     pixel left unreached, is reported as EPIC_ERR_INVALID.
 *   - matches:  float32 [N*4], rows (x, y, x', y').  The source pixel of match
 *     m is (floor(x+0.5), floor(y+0.5)) and must lie inside the image; two
 *     matches may share a source pixel (the smaller index owns it).
 *   - flow_out: float32 [H*W*2], (u, v) = F(p) - p interleaved per pixel.
 *   - At most 4,194,302 matches per pair (22-bit labels).
 *   - Pixel distances are exact fixed-point sums; graph distances and
 *     weighted sums are float32 (sums compensated); the per-match 3x3 normal
 *     equations are solved in float64.
 *   - Ties go to the smallest match index (labels, K-th neighbour).
 *   - All device pointers are caller-owned and must stay valid until the
 *     work enqueued on `stream` has finished.  The handle owns every scratch
 *     buffer (a single device arena, grown on demand).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream-ordered; entry points do not synchronise
 *     unless stated.
 *
 * Errors: every function returns an epic_status_t.  Argument errors are
 * reported immediately; errors found on the device (a match outside the
 * image, a capacity or pass limit) are recorded in a device status word and
 * returned by epic_interp_sync().  epic_interp_last_error() gives a message.
 * A handle is not thread-safe: one host thread at a time.
 */
#ifndef EPIC_INTERP_H
#define EPIC_INTERP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EPIC_OK = 0,
    EPIC_ERR_INVALID = 1,        /* bad argument or bad match coordinate */
    EPIC_ERR_OOM = 2,            /* device or pinned-host allocation failed */
    EPIC_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    EPIC_ERR_NOT_CONVERGED = 4,  /* relaxation hit max_passes */
    EPIC_ERR_TIMEOUT = 5,        /* a bounded grid-barrier wait expired */
    EPIC_ERR_CAPACITY = 6        /* a fixed-capacity structure overflowed
                                    (edge table, node degree, K-NN frontier) */
} epic_status_t;

/* Largest neighbourhood size K of the interpolator, after K is clamped to N
 * (the paper uses K = 100).  A K-NN search keeps its node table (~3.84 K
 * slots), frontier (~1.92 K entries) and settled list in the shared memory
 * of one warp; a search that outgrows them is re-run with tables of 8192
 * node slots, which stay larger than the first tables up to this K.  A run
 * with a larger K returns EPIC_ERR_INVALID; a config max_K above it is
 * treated as EPIC_MAX_K. */
enum { EPIC_MAX_K = 2048 };

typedef struct epic_interp epic_interp_t;

typedef struct {
    int max_H, max_W;     /* largest frame the arena is first sized for */
    int max_N, max_K;     /* largest match count / neighbourhood size
                             (max_K at most EPIC_MAX_K) */
    int max_pairs;        /* largest batch the arena is first sized for */
    int max_passes;       /* cap on relaxation verification passes */
    int weight_squared;   /* 1: Eq. 2 rows scaled by k, i.e. minimise
                             sum k^2 |r|^2 (default); 0: minimise sum k |r|^2 */
    float fallback_eps;   /* fit is degenerate when det M <= eps (tr M/3)^3
                             or fewer than 3 neighbours; then the NW estimate
                             of Eq. 1 at p_m is used as a constant flow */
    int tile_w, tile_h;   /* relaxation tile (0 = 64 x 16 with sweep 2, else
                             64 x 32); with sweep 2 the width is always 64
                             and tile_h at most 32 */
    int apron;            /* sweep 0 / 1: extra context around a tile in the
                             first relaxation pass (-1 = 4); sweep 2: none */
    int keep_intermediates; /* 1: keep K-NN lists for epic_interp_get_knn */
    int max_degree;       /* ignored: the match graph is stored as CSR rows
                             with no degree limit */
    int use_graphs;       /* 1: capture the launch sequence once per table
                             slot and replay it as a CUDA graph (needs a
                             non-default stream, K <= max_K and tiles no
                             larger than the configured ones; otherwise the
                             run uses plain launches) */
    int estimator;        /* 0: locally-weighted affine fit (Eq. 2, default);
                             1: Nadaraya-Watson (Eq. 1), a constant flow per
                             cell (Algorithm 1) */
    int prune;            /* 1: consistency pruning before the interpolation
                             (Sec. 4.1, "Pruning of matches"): a first pass
                             computes the NW estimate at every match with
                             prune_K neighbours, matches whose flow is farther
                             than prune_threshold px from it are removed, and
                             the configured estimator then runs on the kept
                             matches with K neighbours.  If no match of a pair
                             passes, the pair keeps all its matches. */
    float prune_threshold; /* px (default 5) */
    int prune_K;          /* neighbours of the NW pass (default 25) */
    int sweep;            /* relaxation schedule when no tile rule applies
                             (see epic_tile_rule_t; default 2).  The warp
                             tiles of schedule 2 are used only when this and
                             every installed rule ask for them; otherwise a
                             frame whose rule says 2 gets 64 x 32 tiles with
                             apron 4 and schedule 0.  The exact variant's
                             single-source runs always use schedule 0 or 1.
                             Every schedule gives the same result. */
    long long exact_chunk_bytes; /* epic_exact_interp with metric 0: device
                             bytes of packed keys its single-source
                             relaxations may hold at once (8 bytes per pixel
                             per match); the matches run in chunks of
                             max(1, min(N, exact_chunk_bytes / (8 H W))).
                             0 = 1 GiB (default).  Only speed and memory
                             depend on it, never the results. */
} epic_config_t;

/* One frame pair of a batch; pointers are device pointers. */
typedef struct {
    const float *cost_map;  /* [H*W] */
    const float *matches;   /* [N*4] */
    int H, W, N, K;
    float a;
    float *flow_out;        /* [H*W*2] */
} epic_pair_desc_t;

/* A relaxation tile rule: frames of at most max_pixels pixels use tiles of
 * tile_w x tile_h with the given first-pass apron and schedule:
 *   0: a CTA solves a tile with its apron by directional sweeps, lines cut
 *      into segments so every thread of the CTA has one;
 *   1: the same, a thread sweeping whole lines;
 *   2: a warp solves a tile of 64 x tile_h (tile_h 1..32, apron 0) by down
 *      and up passes over its rows, each row taking the three candidates of
 *      the row before it and then closed along itself (the default). */
typedef struct {
    long long max_pixels;
    int tile_w, tile_h, apron;
    int sweep;
} epic_tile_rule_t;

/* Fill *cfg with defaults (sizes for a 1024x436 frame, 5000 matches,
 * K = 100, squared weights, eps = 1e-10, max_passes = 4096). */
void epic_config_default(epic_config_t *cfg);

/* Create a handle on CUDA device `device` and allocate its scratch arena for
 * the sizes in *cfg (NULL = defaults).  Returns EPIC_ERR_OOM if the arena
 * cannot be allocated, EPIC_ERR_CUDA for other runtime failures. */
int epic_interp_create(epic_interp_t **h, int device, const epic_config_t *cfg);

/* Interpolate one pair (Algorithm 1, LA form).  Device pointers; K is
 * clamped to N; requires H, W, N >= 1, K >= 1, min(K, N) <= EPIC_MAX_K and
 * a > 0 (else EPIC_ERR_INVALID, nothing enqueued).  Enqueues the whole path
 * on `stream` and returns without waiting. */
int epic_interp_run(epic_interp_t *h, const float *cost_map,
                    const float *matches, int H, int W, int N, int K, float a,
                    float *flow_out, void *stream);

/* Interpolate n independent pairs of any sizes in one batched launch
 * sequence.  Same rules as epic_interp_run for every descriptor. */
int epic_interp_run_batch(epic_interp_t *h, const epic_pair_desc_t *pairs,
                          int n, void *stream);

/* Same as epic_interp_run but with HOST buffers: copies cost_map and matches
 * to the device, runs, copies the flow back and waits for completion.
 * Returns the device status (as epic_interp_sync would). */
int epic_interp_run_host(epic_interp_t *h, const float *cost_map,
                         const float *matches, int H, int W, int N, int K,
                         float a, float *flow_out, void *stream);

/* Batched form of epic_interp_run_host: every descriptor holds HOST
 * pointers.  Copies all inputs to the device (one cudaMemcpyAsync per
 * buffer; pinned host memory makes them asynchronous DMA), runs the batch,
 * copies every flow back and waits.  Returns the device status. */
int epic_interp_run_batch_host(epic_interp_t *h, const epic_pair_desc_t *pairs,
                               int n, void *stream);

/* Streaming form of epic_interp_run_batch_host, for a sequence of batches
 * with HOST buffers.  Enqueues the batch's uploads, its run and the
 * downloads of its flows, and returns without waiting, so that consecutive
 * calls overlap: a batch's uploads run on a copy stream while the previous
 * batch computes, and its downloads on a second copy stream while the next
 * one computes (the run itself goes on a third, internal stream).  At most
 * two batches are in flight: a third call first waits, on the host, until
 * the downloads of the batch two calls back have finished.  The host buffers
 * must stay valid, and the inputs unchanged, until epic_interp_sync(h)
 * returns; sync waits for every submitted batch and returns the device
 * status.  Pinned host memory is needed for the copies to overlap.  The
 * device staging (two buffers of the batch's inputs and flows) is owned by
 * the handle.  Errors as epic_interp_run_batch. */
int epic_interp_submit_batch_host(epic_interp_t *h, const epic_pair_desc_t *pairs, int n);

/* Wait for the last run's stream (and for every batch submitted with
 * epic_interp_submit_batch_host) and return the device status (then clear
 * it).  EPIC_OK when every stage completed within its limits. */
int epic_interp_sync(epic_interp_t *h);

/* Stage (a) of pair `pair` of the last run: labels L [H*W] int32 and
 * distances D [H*W] float32 (device pointers; either may be NULL). */
int epic_interp_get_labels(epic_interp_t *h, int pair, int *labels_out,
                           float *dist_out, void *stream);

/* Stage (b): number of undirected edges of G of pair `pair` of the last run
 * (waits for the stream). */
int epic_interp_get_edge_count(epic_interp_t *h, int pair, int *n_edges);

/* Stage (b): the edges (m < n, weight) in unspecified order into device
 * buffers of capacity `cap` each; *n_edges receives the count (waits). */
int epic_interp_get_graph(epic_interp_t *h, int pair, int *em, int *en,
                          float *ew, int cap, int *n_edges);

/* Stage (c): K-NN lists of pair `pair` (requires keep_intermediates = 1):
 * idx [N*K] int32 and dist [N*K] float32 in settle order, count [N] int32
 * (device pointers). */
int epic_interp_get_knn(epic_interp_t *h, int pair, int *idx, float *dist,
                        int *count, void *stream);

/* Stage (c): per-match models [N*8] float32 (c_u, c_v, b11, b12, b21, b22,
 * x_m, y_m), flow(p) = c + B (p - p_m); and fallback flags [N] int32
 * (1 = NW fallback).  Device pointers; either may be NULL. */
int epic_interp_get_models(epic_interp_t *h, int pair, float *models,
                           int *fallback, void *stream);

/* Consistency pruning of pair `pair` of the last run (needs prune = 1;
 * waits for the stream).  keep [N] int32: 1 where match m passed the check
 * of Sec. 4.1 (N = the pair's match count as submitted); kept_index
 * [capacity N] int32: the original index of each match the interpolation
 * used, in order (every match when none passed); *n_kept: their number.
 * keep and kept_index are device pointers and may be NULL.  After a pruned
 * run, the labels, graph, K-NN lists and models of the other getters are
 * those of the second pass: match indices there refer to positions in
 * kept_index. */
int epic_interp_get_pruning(epic_interp_t *h, int pair, int *keep,
                            int *kept_index, int *n_kept);

/* Number of relaxation verification passes the last run needed for its
 * whole batch (waits for the stream).  The warp-tile relaxation (schedule 2)
 * has no passes: it reports its tile solves divided by the batch's tile
 * count, rounded up, as equivalent passes. */
int epic_interp_get_passes(epic_interp_t *h, int *passes);

/* Distance unit of pair `pair` of the last run: its keys count distance in
 * units of 2^-(31 - *shift) (waits for the stream).  0 unless the pair's
 * costs reach 2 or its distances could reach 1024 (see the cost range in the
 * conventions above); always 0 with relaxation schedules 0 and 1. */
int epic_interp_get_distance_unit(epic_interp_t *h, int pair, int *shift);

/* Number of matches of the last run whose K-NN search outgrew the per-warp
 * tables of the main pass and was run again with large tables (the final
 * interpolation pass when pruning; waits for the stream).  Diagnostic only:
 * the results do not depend on it, and the retry list holds every match of
 * the batch, so any number of retries succeeds. */
int epic_interp_get_knn_retries(epic_interp_t *h, int *retries);

/* Install relaxation tile rules (replacing any earlier ones; n = 0 clears
 * them).  A pair uses the first rule whose max_pixels >= H*W, else the
 * configured tile.  Tile sides must be in [8, 256], apron < min(side) and
 * <= 64.  Rules only change speed, never results (every tiling reaches the
 * same fixed point).  The rules are copied. */
int epic_interp_set_tile_rules(epic_interp_t *h, const epic_tile_rule_t *rules,
                               int n);

/* Stage timing.  While enabled, every run records CUDA events on its
 * stream around its stages: 0 prepare, 1 relaxation, 2 edges, 3 scatter (CSR
 * offsets and rows, the lightest edges per node, the K-NN bound edges),
 * 4 K-NN + fit, 5 write-out, 6 pruning (the whole first pass and the
 * compaction; zero when prune = 0).  Enabling (again) clears the
 * accumulated times. */
int epic_interp_enable_stage_timing(epic_interp_t *h, int enable);

/* Sum over the runs since timing was enabled of each stage's elapsed time in
 * milliseconds, into ms_out[0..n_stages) (n_stages <= 7); *n_runs receives
 * the number of runs summed.  Waits for the last timed run. */
int epic_interp_get_stage_times(epic_interp_t *h, float *ms_out, int n_stages,
                                int *n_runs);

/* Exact variant (Sec. 5.2, Table 2): every pixel p takes its own K nearest
 * matches under the exact distance, keyed (distance, index), and its own fit
 * (Eq. 2 centred at p, or the NW estimate of Eq. 1 with estimator = 1; a
 * degenerate fit falls back to NW as in the main path).  The flow at p is
 * the model's value at p.  metric 0: the geodesic distance D_G of Eq. 3,
 * computed by one single-source relaxation per match (the paper's "exact"
 * geodesic row).  Each relaxation is capped where its match cannot be among
 * a pixel's K nearest: an approximate run on the same handle (its K-NN
 * lists; it replaces the handle's last-run state) bounds every match's K-th
 * nearest distance, and a relaxation seeded with those bounds gives a
 * 1-Lipschitz upper bound of every pixel's K-th nearest distance; distances
 * beyond it are not needed and not computed.  metric 1: the Euclidean
 * distance between pixel centres and
 * match pixels (the paper's "Euclidean" row).  Device pointers; cost_map,
 * matches and flow_out as for epic_interp_run; knn_idx_out [H*W*K] int32 and
 * knn_dist_out [H*W*K] float32 receive every pixel's list in key order (both
 * NULL, or both set).  K is clamped to N and limited by shared memory
 * (K * 512 bytes per 64 pixels; K <= 448 on GB300).  With metric 0 the
 * handle holds N * H * W * 4 bytes of distances plus up to
 * exact_chunk_bytes (1 GiB by default) of relaxation keys (grown on demand,
 * EPIC_ERR_OOM if it cannot be).  Runs
 * on `stream` and waits for completion; returns the device status. */
int epic_exact_interp(epic_interp_t *h, const float *cost_map,
                      const float *matches, int H, int W, int N, int K,
                      float a, int metric, float *flow_out, int *knn_idx_out,
                      float *knn_dist_out, void *stream);

/* Cost map from an image (Table 2, the "||grad_2 I||_2" contour row, a
 * stand-in for a learned edge detector): for each of `frames` images
 * [H][W][channels] float32 (interleaved channels, values in [0, 1],
 * frames stored back to back), cost_out [frames][H][W] receives
 *   C(p) = floor + sqrt(sum_c gx_c^2 + gy_c^2),
 * gx = (I(x+1) - I(x-1)) / 2 and gy likewise, on the image padded by edge
 * replication (each frame's borders are its own).  With values in [0, 1]
 * C - floor <= sqrt(channels / 2), inside the interpolator's [0, 2) for up
 * to 3 channels when floor < 0.77.  channels = 1, 3 or 4; floor finite and
 * >= 0.  Device pointers on the current device; enqueued on `stream`
 * without waiting.  Needs no handle. */
int epic_gradient_cost(const float *image, int frames, int H, int W,
                       int channels, float floor, float *cost_out,
                       void *stream);

/* Variational refinement (Sec. 4, "Variational Energy Minimization").  The
 * paper fixes the structure: a data term with colour and gradient constancy
 * and a normalisation factor, a smoothness term on the flow gradient with
 * local weight alpha(x) = alpha0 exp(-kappa ||grad I1(x)||), kappa = 5, and
 * a full-resolution minimisation by `iterations` (5) fixed-point iterations
 * with `sor_iterations` (30) SOR iterations per linear system.  The
 * remaining constants are this library's defaults: gamma (weight of the
 * gradient term) 0.7, robust penaliser sqrt(s^2 + eps^2) with eps 1e-3,
 * normalisation 1 / (|grad|^2 + zeta^2) with zeta 0.1, alpha0 1, SOR
 * relaxation omega 1.6. */
typedef struct {
    float alpha0, gamma, kappa, eps, zeta, omega;
    int iterations, sor_iterations;
} epic_refine_params_t;

void epic_refine_params_default(epic_refine_params_t *p);

/* Refine flow [H*W*2] in place between images I1 and I2 [H*W*channels]
 * float32 (interleaved channels, values in [0, 1]; channels 1..4).  Each
 * fixed-point iteration warps I2 by the current flow (bilinear, clamped
 * coordinates), linearises the data term there with the robust weights
 * taken at zero update, and solves for the update with red-black SOR in
 * which each pixel's 2x2 (du, dv) system is solved exactly; derivatives are
 * central differences on edge-replicated images.  Device pointers (flow
 * 8-byte aligned, else EPIC_ERR_INVALID); the
 * handle holds about H*W*(channels + 12)*4 bytes of scratch (grown on demand,
 * EPIC_ERR_OOM if it cannot be).  Enqueued on `stream` without waiting; one
 * refinement in flight per handle (the scratch is shared).  params NULL =
 * defaults. */
int epic_refine(epic_interp_t *h, const float *I1, const float *I2, int H,
                int W, int channels, float *flow,
                const epic_refine_params_t *params, void *stream);

/* Self-test of failure detection without a GPU fault.  Every device wait
 * of the library is bounded: the relaxation's grid barrier (2 s) and the TMA
 * staging's mbarrier wait (1 s) give up, record EPIC_ERR_TIMEOUT and let the
 * kernel return.  This runs one of those waits with a limit of limit_ms
 * (1..10000) where the awaited event never happens: which = 0, a grid
 * barrier that expects a second CTA which does not exist; which = 1, an
 * mbarrier whose transaction is never issued.  Returns the status the wait
 * recorded (EPIC_ERR_TIMEOUT when the bound works) and leaves the handle and
 * the context usable.  Waits for completion. */
int epic_selftest_wait_timeout(epic_interp_t *h, int which, int limit_ms);

/* Device scratch one pair of H x W pixels, N matches and neighbourhood size
 * K takes in the handle's arena when it runs in a batch (its packed keys,
 * seed bins, edge table, CSR rows, models, optional K-NN lists and pruning
 * buffers, its K-NN retry-list slots and its relaxation tiles' work-queue
 * slots), in *bytes; a batch needs the sum over its pairs plus 512 bytes.  The caller's own buffers (cost map,
 * matches, flow) are not included.  Uses the configuration and tile rules of
 * `h`; with h = NULL, those of *cfg and no tile rules (cfg = NULL: the
 * defaults).  A host computation: needs no device and enqueues nothing.
 * EPIC_ERR_INVALID for sizes that epic_interp_run would refuse. */
int epic_interp_request_bytes(const epic_interp_t *h, const epic_config_t *cfg, int H,
                              int W, int N, int K, long long *bytes);

/* Number of kernel launches one run of `n` pairs enqueues. */
int epic_interp_launches_per_run(epic_interp_t *h, int n);

/* Stage (a) alone -- the assignment map L and distance D -- computed without
 * allocating any device memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot let a library allocate, such as a
 * host framework that owns every device allocation and only lends buffers,
 * or a latency-critical loop where cudaMalloc's implicit synchronisation is
 * not acceptable.  Inputs as for epic_interp_run (device pointers, matches
 * 16-byte aligned); outputs labels_out [H*W] int32 and dist_out [H*W]
 * float32 (device pointers, either may be NULL but not both), identical to
 * epic_interp_get_labels after epic_interp_run.
 *   - Scratch is a file-scope device array of the library (about 5 MB, held
 *     by every GPU that loads the library until the process exits); frames
 *     are limited to 524288 pixels, 32768 matches and 16384 relaxation tiles
 *     of 64 x 32 pixels.  Larger inputs return EPIC_ERR_CAPACITY without
 *     doing any work.
 *   - Runs on the current device.  Every call looks up the array's device
 *     address in the current CUDA context (cudaGetSymbolAddress, a host-side
 *     query), so a context reset between calls is harmless.  The first call
 *     in a context may load the library's device code; make that first call
 *     before any stream capture.
 *   - The small argument blocks (one pair descriptor, its prefix sums, the
 *     launch arguments) are copied into the array by cudaMemcpyAsync from
 *     the call's own stack; a copy from pageable host memory has read its
 *     source by the time cudaMemcpyAsync returns.
 *   - Every call shares the array: calls that overlap on the GPU race.  Each
 *     call clears its run state, waits for its own work on `stream` and
 *     returns the device status (EPIC_OK, or e.g. EPIC_ERR_INVALID for a
 *     match outside the image). */
int epic_geodesic_labels_noalloc(const float *cost_map, const float *matches,
                                 int H, int W, int N, int *labels_out,
                                 float *dist_out, void *stream);

/* Message describing the last error on this handle (never NULL). */
const char *epic_interp_last_error(epic_interp_t *h);

/* Release the arena and the handle (waits for outstanding work). */
void epic_interp_destroy(epic_interp_t *h);

#ifdef __cplusplus
}
#endif

#endif /* EPIC_INTERP_H */
