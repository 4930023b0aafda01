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

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/epic_interp.h"

namespace epic {

// Packed (distance, label) key of the geodesic relaxation.  The high word is
// the IEEE-754 bit pattern of a non-negative float32 distance, whose unsigned
// order equals numeric order; the low word is the match index.  Comparing
// keys as uint64 therefore compares (D, L) lexicographically, which realises
// "nearest match, ties to the smallest index" (Sec. 3.4), and a 64-bit access
// moves both halves at once so no reader ever sees a torn pair.
typedef unsigned long long pkey_t;
constexpr pkey_t KEY_INF = 0x7F800000FFFFFFFFull;  // (+inf, no label)
constexpr unsigned EMPTY32 = 0xFFFFFFFFu;
constexpr pkey_t EMPTY64 = 0xFFFFFFFFFFFFFFFFull;

__device__ __forceinline__ pkey_t make_key(float d, unsigned label) {
    return ((pkey_t)__float_as_uint(d) << 32) | label;
}
__device__ __forceinline__ float key_dist(pkey_t k) {
    return __uint_as_float((unsigned)(k >> 32));
}
__device__ __forceinline__ unsigned key_label(pkey_t k) { return (unsigned)k; }

// Step cost of Eq. 3 between 8-neighbours p, q, from half-costs
// h = C/2: |p-q| (C(p)+C(q))/2 = |p-q| (h(p)+h(q)).  Multiplying by 1/2 is
// exact in float32, so h(p)+h(q) == (C(p)+C(q))/2 bit for bit.  Explicit
// round-to-nearest intrinsics keep the compiler from contracting the
// product into a later addition, so every kernel evaluates the identical
// float32 value for the same step.
constexpr float SQRT2_F = 1.41421356237309515f;
__device__ __forceinline__ float step_axis(float hp, float hq) {
    return __fadd_rn(hp, hq);
}
__device__ __forceinline__ float step_diag(float hp, float hq) {
    return __fmul_rn(SQRT2_F, __fadd_rn(hp, hq));
}

// Per-pair state; every pointer is a device address.
struct PairDev {
    const float *C;         // [H*W] caller's cost map
    const float4 *matches;  // [N] (x, y, x', y') caller's matches
    float *flow;            // [H*W*2] caller's output
    int H, W, N, K;
    float a;
    int tile_w, tile_h, apron;
    int tiles_x, tiles_y;
    int hash_cap;           // power of two
    int flow_vec_ok;        // flow pointer is 16-byte aligned
    pkey_t *keys;            // [H*W] packed (D, L)
    int *tile_start;        // [tiles+1] seed bins (prefix offsets)
    int *tile_fill;         // [tiles] scatter cursors
    int *tile_seeds;        // [N] match indices grouped by tile
    int *tile_stamp;        // [tiles] last relaxation pass that wrote the tile
    pkey_t *hkeys;           // [hash_cap] (m << 32 | n), m < n
    unsigned *hw;           // [hash_cap] float bits of the edge weight
    int *deg;               // [N] node degree in G
    unsigned *wmin;         // [N] float bits of the lightest edge at each node
    pkey_t *adj;             // [N * max_degree] (w bits << 32 | neighbour)
    float4 *models;         // [N * 2] (c_u, c_v, b11, b12), (b21, b22, x_m, y_m)
    int *fallback;          // [N]
    int *knn_idx;           // [N*K] or null
    float *knn_dist;        // [N*K] or null
    int *knn_count;         // [N] or null
    int *info;              // [4] edges, max degree, spare
};

struct GridBarrier {
    unsigned count;
    unsigned gen;
};

// Counters that live in the arena for the whole handle.
struct RunState {
    int status;            // first device error (epic_status_t), 0 = OK
    int passes;            // relaxation verification passes of the last run
    unsigned changed[3];   // per-pass dirty-tile counters (rotating)
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
    int max_degree;
    int knn_hs, knn_fs, knn_kmax;  // per-warp K-NN table sizes (powers of 2) and K bound
    int max_passes;
    int weight_squared;
    float fallback_eps;
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
};
// Launchers: `a` is the host copy of the launch arguments (used only for
// launch-shape decisions), `dev` the same struct in device memory (the
// kernels' only parameter, so a captured launch sequence can be replayed for
// any batch whose table has been uploaded to the same address).
cudaError_t launch_prepare(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc);
cudaError_t launch_dt(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc,
                      int max_tile_w, int max_tile_h, int max_apron, bool fixed_grid,
                      int *grid_used);
cudaError_t launch_edges(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc);
cudaError_t launch_scatter(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc);
cudaError_t launch_knn_fit(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc,
                           int max_K);
cudaError_t launch_writeout(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc);
cudaError_t launch_split_keys(const PairDev *pair_host_copy, int *labels,
                              float *dist, cudaStream_t stream);
cudaError_t launch_collect_edges(const PairDev *pair_host_copy, int *em,
                                 int *en, float *ew, int cap, int *count,
                                 cudaStream_t stream);
size_t dt_smem_bytes(int tile_w, int tile_h, int apron);
void knn_table_sizes(int max_K, int *hs, int *fs);
size_t knn_smem_per_warp(int max_K);
int knn_warps_per_cta(int max_K, int smem_limit);

}  // namespace epic
