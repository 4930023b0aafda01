// Internal device-side structures shared by the interpolator's kernels.
//
// A run processes a batch of independent frame pairs.  The host lays out one
// PairDev per pair (pointers into the handle's arena plus the caller's
// buffers) and uploads the table together with prefix sums that map a flat
// work index (tile, match, pixel chunk, hash slot) back to its pair.  Every
// kernel is launched with a fixed, SM-count-derived grid and walks its flat
// work range with a grid-stride loop, so the launch shape never depends on
// the batch contents.
#pragma once

#include <cuda.h>            // CUtensorMap (type only; no driver library is linked)
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/epic_interp.h"

namespace epic {

// Packed (distance, label) key of the geodesic relaxation.
//   bit 63       : unreached flag
//   bits 62..22  : D in fixed point, units of 2^-31 (D < 2^41 units = 1024)
//   bits 21..0   : match index (label), 0x3FFFFF = none
// Comparing keys as uint64 compares (D, L) lexicographically, which realises
// "nearest match, ties to the smallest index" (Sec. 3.4), and a 64-bit access
// moves both halves at once so no reader ever sees a torn pair.  Path sums
// are integers, hence exact and associative: the minimum key over all paths
// is then the unique fixed point of the relaxation whatever order the steps
// run in (with rounded float sums, a step absorbed by rounding can leave a
// label that depends on the order).  A step adds (w << 22) to the
// neighbour's key, carrying its label along.
typedef unsigned long long pkey_t;
constexpr int LABEL_BITS = 22;
constexpr unsigned LABEL_NONE = (1u << LABEL_BITS) - 1u;
constexpr pkey_t KEY_INF = 0x8000000000000000ull | LABEL_NONE;
constexpr unsigned EMPTY32 = 0xFFFFFFFFu;
constexpr pkey_t EMPTY64 = 0xFFFFFFFFFFFFFFFFull;
constexpr int MAX_LABELS = (1 << LABEL_BITS) - 2;    // largest N
constexpr float UNITS_PER_ONE = 2147483648.0f;        // 2^31
constexpr float ONE_PER_UNIT = 4.6566128730773926e-10f;  // 2^-31

__device__ __forceinline__ pkey_t make_key(unsigned long long d_units, unsigned label) {
    return (d_units << LABEL_BITS) | label;
}
__device__ __forceinline__ unsigned long long key_dunits(pkey_t k) { return k >> LABEL_BITS; }
__device__ __forceinline__ bool key_reached(pkey_t k) { return !(k >> 63); }
__device__ __forceinline__ float key_dist(pkey_t k) {
    return key_reached(k) ? __fmul_rn(__ull2float_rn(key_dunits(k)), ONE_PER_UNIT)
                          : __int_as_float(0x7f800000);
}
__device__ __forceinline__ unsigned key_label(pkey_t k) { return (unsigned)k & LABEL_NONE; }

// Step cost of Eq. 3 between 8-neighbours p, q in fixed-point units:
// |p-q| (C(p)+C(q))/2 = |p-q| (h(p)+h(q)) with half-costs h = C/2 held as
// integers h = rint(C 2^30) (units of 2^-31; 0 <= C < 2).  An axis step is
// the exact sum of the two halves; a diagonal step multiplies that sum by
// sqrt 2 in 2.30 fixed point, rounded to the nearest unit.  Both are
// symmetric in p, q and every kernel forms the identical integer.
constexpr float C_MAX = 2.0f;  // costs are edge strengths in [0, 2)
constexpr unsigned long long SQRT2_Q30 = 1518500250ull;  // rint(sqrt(2) 2^30)
__device__ __forceinline__ unsigned step_axis(unsigned hp, unsigned hq) {
    return hp + hq;   // < 2^32: half-costs are below 2^31
}
__device__ __forceinline__ unsigned long long step_diag(unsigned hp, unsigned hq) {
    return ((unsigned long long)(hp + hq) * SQRT2_Q30 + (1ull << 29)) >> 30;
}
// h = rint(C 2^30) for 0 <= C < C_MAX, else 0 and *bad set.
__device__ __forceinline__ unsigned half_cost(float c, bool *bad) {
    if (!(c >= 0.f && c < C_MAX)) {
        *bad = true;
        return 0u;
    }
    return __float2uint_rn(__fmul_rn(c, 1073741824.0f));
}
// Per-pair distance unit of the warp-tile relaxation.  A pair's keys count
// distance in units of 2^-(31 - s) and its half-costs are
// h = rint(C 2^(30 - s)), so costs up to 2^(1 + s) and distances up to
// 2^(10 + s) fit; s = 0 (the unit above) unless the pair needs more.  The
// prepare kernel records the pair's largest cost (cmax_bits) and how many
// tile steps separate the farthest tile from a tile holding a seed
// (seed_reach); every pixel then lies within an octile distance of
// (reach + 1) (max(tw, th) + (sqrt 2 - 1) min(tw, th)) pixels of a seed, and
// its geodesic distance is at most the largest cost times that.  Every kernel
// derives s from these two fields with this function, so they agree.
constexpr int STAMP_PENDING = (int)0x80000000;   // a warp tile not yet written this run
constexpr int MAX_UNIT_SHIFT = 20;
constexpr int SWEEP_WARP = 2;   // relaxation schedule of the warp tiles
__host__ __device__ __forceinline__ int unit_shift_of(unsigned cmax_bits, int reach, int tw,
                                                      int th) {
    if (cmax_bits > 0x7f800000u) return 0;   // NaN or negative: reported as an invalid cost
    float cmax;
    memcpy(&cmax, &cmax_bits, sizeof cmax);
    const float r = (float)(reach + 1);
    const float ext = r * (float)(tw > th ? tw : th) + 0.41421357f * r * (float)(tw < th ? tw : th);
    const float dbound = cmax * ext * 1.001f + 1e-3f;
    int s = 0;
    while (s < MAX_UNIT_SHIFT && (cmax >= ldexpf(2.f, s) || dbound >= ldexpf(1024.f, s))) ++s;
    return s;
}
// h = rint(C 2^(30 - s)) for 0 <= C < C_MAX 2^s, else 0 and *bad set.
__device__ __forceinline__ unsigned half_cost_s(float c, int s, bool *bad) {
    if (!(c >= 0.f && c < ldexpf(C_MAX, s))) {
        *bad = true;
        return 0u;
    }
    return __float2uint_rn(__fmul_rn(c, ldexpf(1073741824.0f, -s)));
}
// Distance of `units` fixed-point units of shift s, rounded once to float32.
__device__ __forceinline__ float units_dist(unsigned long long units, int s) {
    return __fmul_rn(__ull2float_rn(units), ldexpf(ONE_PER_UNIT, s));
}

// Candidate key at p from neighbour key kq over a step of w units; an
// unreached neighbour offers nothing (its flag bit makes the sum >= KEY_INF).
__device__ __forceinline__ pkey_t step_key(pkey_t kq, unsigned long long w) {
    return kq + (w << LABEL_BITS);
}

// Per-pair state; every pointer is a device address.
struct PairDev {
    const float *C;         // [H*W] caller's cost map
    const float4 *matches;  // [N] (x, y, x', y') caller's matches
    float *flow;            // [H*W*2] caller's output
    int H, W, N, K;
    float a;
    int tile_w, tile_h, apron;
    int sweep;              // relaxation schedule: 0 segmented lines, 1 whole lines
                            // (k_dt.cu); 2 row-closure passes on warp tiles (k_relax.cu)
    int tiles_x, tiles_y;
    int hash_cap;           // power of two
    int flow_vec_ok;        // flow pointer is 16-byte aligned
    pkey_t *keys;            // [H*W] packed (D, L)
    // exact variant only (null elsewhere): a distance offset per seed (units),
    // and a key map whose distances cap the keys written back (a pixel whose
    // distance exceeds its cap is left unreached)
    const unsigned long long *seed_init;   // [N]
    const pkey_t *cap;                     // [H*W]
    int *tile_start;        // [tiles+1] seed bins (prefix offsets)
    int *tile_fill;         // [tiles] scatter cursors
    int *tile_seeds;        // [N] match indices grouped by tile
    int *tile_stamp;        // [tiles] last relaxation pass that wrote the tile
                            // (STAMP_PENDING: not yet in this run; warp tiles)
    pkey_t *hkeys;           // [hash_cap] (m << 32 | n), m < n
    unsigned *hw;           // [hash_cap] float bits of the edge weight
    int *deg;               // [N] node degree in G, then the CSR fill cursor
    unsigned *wmin;         // [N] float bits of the lightest edge at each node
    unsigned *wmin2;        // [N] float bits of the second-lightest edge (+inf if none)
    int *wnear;             // [N] other end of the lightest edge (-1 if none)
    int *row;               // [N + 1] CSR row offsets into adj
    uint4 *adj;              // [2 * hash_cap] CSR rows: (neighbour, w bits, the
                             // neighbour's lightest-edge bits, 0)
    float4 *models;         // [N * 2] (c_u, c_v, b11, b12), (b21, b22, x_m, y_m)
    int *fallback;          // [N]
    int *knn_idx;           // [N*K] or null
    float *knn_dist;        // [N*K] or null
    int *knn_count;         // [N] or null
    int *info;              // [4] edges, max degree, spare
    // consistency pruning (Sec. 4.1 "Pruning of matches"): the first pass
    // writes keep[N]; the compaction rewrites matches/N/K of this entry in
    // device memory for the second pass
    int *keep;              // [N] 1 = kept, or null when not pruning
    float4 *pruned;         // [N] kept matches, in their original order
    int *kept_index;        // [N] original index of each kept match
    int K2;                 // K of the second (LA) pass
    // TMA staging of the relaxation's cost tiles (tma_cost = 0: plain loads):
    // 2D tensor maps over C (W x H float32) with boxes of (bw, RH) for the
    // phase-1 region (tile + apron + ring) and the re-solve region (tile +
    // ring); bw covers the region from its x origin rounded down to a
    // multiple of 4, as TMA requires 16-byte-aligned x coordinates.
    int tma_cost;
    int tma_bw_fresh, tma_bw_again;
    CUtensorMap tm_cost_fresh;
    CUtensorMap tm_cost_again;
    // TMA staging of the warp tiles (k_relax.cu; tma_warp = 0: plain loads):
    // boxes of the keys (u64, 68 x (tile_h + 2) from x0 - 2) and of the
    // costs (float32, 72 x (tile_h + 2) from x0 - 4), tile and ring
    int tma_warp;
    // written on the device by the prepare kernel (zero from the host): the
    // float bits of the pair's largest cost and the tile-step reach of its
    // seeds, from which unit_shift() derives the distance unit
    unsigned cmax_bits;
    int seed_reach;
    CUtensorMap tm_warp_keys;
    CUtensorMap tm_warp_cost;
};

// The distance unit shift of a pair (0 for the sweep schedules of k_dt.cu,
// which keep the unit 2^-31).
__device__ __forceinline__ int unit_shift(const PairDev &P) {
    return P.sweep == SWEEP_WARP
               ? unit_shift_of(*(volatile const unsigned *)&P.cmax_bits,
                               *(volatile const int *)&P.seed_reach, P.tile_w, P.tile_h)
               : 0;
}

struct GridBarrier {
    unsigned count;
    unsigned gen;
};

// Counters that live in the arena for the whole handle.
struct RunState {
    int status;            // first device error (epic_status_t), 0 = OK
    int passes;            // relaxation verification passes of the last run
    unsigned changed[3];   // per-pass dirty-tile counters (rotating)
    unsigned work[4];      // relaxation tile dispensers: passes (rotating), phase 1
    unsigned knn_next;     // K-NN match dispenser
    unsigned knn_overflow; // matches whose search outgrew the small tables
    unsigned knn_retry;    // dispenser of the retry pass over those matches
    unsigned edge_next;    // boundary-edge tile dispenser
    unsigned wl_count[3];  // worklist lengths of the chunked relaxation passes (rotating)
    unsigned compact_done; // CTAs finished in the pruning compaction
    // the warp-tile relaxation's work queue (phase 2): tickets taken, items
    // pushed, items pushed or held but not finished, items taken
    unsigned q_head, q_tail;
    int q_busy;
    unsigned q_items;
    GridBarrier barrier;
};

// Launch-wide parameters (passed by value).
struct BatchArgs {
    const PairDev *pairs;
    int npairs;
    const int *tile_base;    // [npairs+1] prefix of tiles
    const int *match_base;   // [npairs+1] prefix of matches
    const int *chunk_base;   // [npairs+1] prefix of write-out chunks
    const int *hash_base;    // [npairs+1] prefix of hash slots
    const int *clear_base;   // [npairs+1] prefix of clear chunks
    int total_tiles, total_matches, total_chunks, total_hash, total_clear;
    int uniform_tiles;       // > 0: every pair has this many tiles (pair = tile / uniform_tiles)
    int *wl;                 // chunked relaxation only: 3 worklists of total_tiles flat tile indices
    int *wl_queued;          // [total_tiles] last pass + 1 a tile was queued for (0 = never)
    int max_degree;
    int knn_hs, knn_fs, knn_kmax;  // main-pass K-NN table sizes per warp, and K bound
    int *relax_queue;      // [total_tiles] warp-tile relaxation work queue (-1 = empty slot);
                           // null for runs of the apron-tile relaxation
    int *relax_queued;     // [total_tiles] per-tile queue state (see k_relax.cu)
    int *knn_retry_list;   // global match indices to search again; holds every match of
                           // the batch (a match is queued at most once per pass)
    int max_passes;
    int weight_squared;
    float fallback_eps;
    int estimator;          // 0 = LA (Eq. 2), 1 = Nadaraya-Watson (Eq. 1)
    int final_estimator;    // estimator of the second pass when pruning
    int write_keep;         // first pass of a pruned run: write PairDev::keep
    float prune_threshold;  // px; a match farther than this from the NW estimate is dropped
    RunState *state;
};

// Which pair does flat index i of a prefix array belong to (largest p with
// base[p] <= i); the arrays are short (one entry per pair).
__device__ __forceinline__ int find_pair(const int *base, int n, int i) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void set_status(RunState *s, int code) {
    atomicCAS(&s->status, 0, code);
}
__device__ __forceinline__ int get_status(const RunState *s) {
    return *(volatile const int *)&s->status;
}

// ---------------------------------------------------------------------------
// Bounded grid barrier of the cooperative relaxation launches.
// ---------------------------------------------------------------------------
constexpr unsigned long long BARRIER_LIMIT_NS = 2000000000ull;  // 2 s
constexpr int PASS_CHUNK = 8;  // tiles per dispenser step in chunked verification passes

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sense-free generation barrier over all CTAs of a cooperative launch.  The
// wait gives up after BARRIER_LIMIT_NS (or as soon as another CTA has given
// up) and reports EPIC_ERR_TIMEOUT instead of spinning forever.
static __device__ __noinline__ bool grid_sync(RunState *st, unsigned nblocks,
                          unsigned long long limit_ns = BARRIER_LIMIT_NS) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        GridBarrier *b = &st->barrier;
        int ok = 1;
        unsigned g = ld_acquire(&b->gen);
        __threadfence();
        unsigned arrived = atomicAdd(&b->count, 1u);
        if (arrived == nblocks - 1) {
            b->count = 0;
            __threadfence();
            st_release(&b->gen, g + 1);
        } else {
            unsigned long long t0 = global_ns();
            while (ld_acquire(&b->gen) == g) {
                if (get_status(st) == EPIC_ERR_TIMEOUT) { ok = 0; break; }
                if (global_ns() - t0 > limit_ns) {
                    set_status(st, EPIC_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

constexpr int WRITEOUT_CHUNK = 1024;  // pixels per write-out work item
constexpr int CLEAR_CHUNK = 4096;     // 8-byte words per clear work item
constexpr int DT_THREADS = 256;
constexpr int KNN_WARPS = 8;          // warps (= matches in flight) per CTA
constexpr int EDGE_THREADS = 256;

// Host-side launchers (one per kernel file).
struct LaunchCfg {
    int num_sms;
    int smem_optin;  // max dynamic shared memory per CTA (opt-in)
    cudaStream_t stream;
    int smem_per_sm = 0;    // shared memory per SM (0: unknown)
    int smem_reserved = 0;  // shared memory the system reserves per CTA
};
// Launchers: `a` is the host copy of the launch arguments (used only for
// launch-shape decisions), `dev` the same struct in device memory (the
// kernels' only parameter, so a captured launch sequence can be replayed for
// any batch whose table has been uploaded to the same address).
cudaError_t launch_prepare(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc);
// chunked_passes: the verification passes hand out tiles in chunks (for
// single-source runs, which need dozens of passes); see dt_kernel.
cudaError_t launch_dt(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc,
                      int max_tile_w, int max_tile_h, int max_apron, bool fixed_grid,
                      int *grid_used, bool chunked_passes = false);
cudaError_t launch_edges(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc,
                         int max_tile_w, int max_tile_h);
cudaError_t launch_scatter(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc);
cudaError_t launch_knn_fit(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc,
                           int max_K);
cudaError_t launch_writeout(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc);
cudaError_t launch_compact(const BatchArgs &a, BatchArgs *dev, const LaunchCfg &lc);

// Exact variant (per-pixel K nearest and fit).
constexpr int EXACT_THREADS = 64;
struct ExactArgs {
    const float *D;          // [N][H*W] distances, or null: Euclidean
    const float4 *matches;   // [N]
    float *flow;             // [H*W*2]
    int *knn_idx;            // [H*W*K] or null
    float *knn_dist;         // [H*W*K] (with knn_idx)
    int *fallback;           // [H*W] or null
    int H, W, N, K;
    float a, fallback_eps;
    int weight_squared, estimator;
};
size_t exact_smem_bytes(int K);
cudaError_t launch_cap_seed(const float *knn_dist, const int *knn_count, int N, int K, int ld,
                            unsigned long long *init, cudaStream_t stream);
cudaError_t launch_keys_to_dist(const pkey_t *keys, long long n, float *D, cudaStream_t stream);
cudaError_t launch_exact_fit(const ExactArgs &x, cudaStream_t stream);

// Self-test of the bounded device waits (grid barrier, TMA mbarrier).
cudaError_t launch_wait_selftest(RunState *st, int which, unsigned long long limit_ns,
                                 cudaStream_t stream);

// Variational refinement.
struct RefineArgs {
    float alpha0, gamma, kappa, eps, zeta, omega;
    int iterations, sor_iterations;
};
size_t refine_scratch_bytes(int H, int W, int C);
cudaError_t launch_refine(const float *I1, const float *I2, int H, int W, int C, float *flow,
                          const RefineArgs &r, void *scratch, int num_sms, cudaStream_t stream);

// Image-gradient cost map.
cudaError_t launch_gradcost(const float *img, int F, int H, int W, int channels, float floor_,
                            float *C, int num_sms, cudaStream_t stream);
// labels / distances of one pair's keys; pair_dev is the pair's device
// descriptor (its distance unit is recorded there on the device)
cudaError_t launch_split_keys(const PairDev *pair_host_copy, const PairDev *pair_dev,
                              int *labels, float *dist, cudaStream_t stream);
cudaError_t launch_collect_edges(const PairDev *pair_host_copy, int *em,
                                 int *en, float *ew, int cap, int *count,
                                 cudaStream_t stream);
size_t dt_smem_bytes(int tile_w, int tile_h, int apron);
// The interpolator's relaxation on warp-owned tiles of 64 x tile_h pixels
// (k_relax.cu); max_rows = the largest tile_h of the batch (<= 32).
constexpr int RELAX_TILE_W = 64;
constexpr int RELAX_MAX_ROWS = 32;
size_t relax_smem_bytes(int max_rows);
cudaError_t launch_relax(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc,
                         int max_rows, bool fixed_grid, int *grid_used);
void knn_table_sizes(int max_K, const LaunchCfg &lc, int *hs, int *fs);
void knn_retry_table_sizes(int max_K, int smem_limit, int *hs, int *fs);
size_t knn_smem_per_warp(int max_K, const LaunchCfg &lc);
int knn_warps_per_cta(int max_K, const LaunchCfg &lc);

}  // namespace epic
