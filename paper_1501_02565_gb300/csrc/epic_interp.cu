// C ABI of the interpolator: handle, scratch arena, batch tables, launches.
//
// A run enqueues, on the caller's stream:
//   table upload (pinned staging -> device), prepare, relaxation
//   (cooperative, all passes in one launch), edge insertion, adjacency
//   scatter, K-NN + fit, write-out.
// The handle owns one device arena that is carved per run into every pair's
// scratch (keys, seed bins, edge table, adjacency, models, optional K-NN
// lists); it grows (after waiting for earlier work) when a batch needs more.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "epic_internal.cuh"

using epic::BatchArgs;
using epic::PairDev;
using epic::RunState;
using epic::pkey_t;

struct epic_interp;
using Handle = epic_interp;

struct epic_interp {
    int device = 0;
    int num_sms = 0;
    int smem_optin = 0;
    int smem_per_sm = 0, smem_reserved = 0;
    epic_config_t cfg{};
    char *arena = nullptr;
    size_t arena_bytes = 0;
    RunState *state = nullptr;      // device
    RunState *state_host = nullptr; // pinned mirror for reads
    int *scratch_count = nullptr;   // device int for getters
    // two batch-table slots used alternately: pinned staging, device copy,
    // the event that marks the slot's last run finished, and (graph mode)
    // the captured launch sequence that reads this slot
    struct Slot {
        char *dev = nullptr;
        char *host = nullptr;
        cudaEvent_t done = nullptr;
        bool pending = false;
        cudaGraphExec_t graph = nullptr;
    } slot[2];
    int next_slot = 0;
    size_t table_cap = 0;
    std::vector<PairDev> pairs;     // last run's descriptors
    const PairDev *pairs_dev = nullptr;  // last run's device descriptors
    bool pruned = false;            // last run pruned (device N, K changed)
    std::vector<int> n_submitted;   // last run's match counts as submitted
    cudaStream_t last_stream = nullptr;
    // streaming host batches (epic_interp_submit_batch_host): internal
    // streams for uploads, runs and downloads, and two staging buffers used
    // alternately, each with the events of its batch's three phases
    cudaStream_t st_up = nullptr, st_run = nullptr, st_down = nullptr;
    struct HostSlot {
        char *buf = nullptr;
        size_t cap = 0;
        cudaEvent_t up = nullptr, ran = nullptr, down = nullptr;
        bool busy = false;
    } hslot[2];
    int next_hslot = 0;
    // device staging for epic_interp_run_host
    float *io_C = nullptr, *io_M = nullptr, *io_F = nullptr;
    size_t io_C_n = 0, io_M_n = 0, io_F_n = 0;
    // scratch of the exact variant (distance rows, relaxation chunk, tables)
    char *ex_buf = nullptr;
    size_t ex_cap = 0;
    // scratch of the variational refinement
    void *rf_buf = nullptr;
    // set by the exact variant around its internal approximate run: keep the
    // K-NN lists, plain launches, no pruning
    bool force_keep = false;
    size_t rf_cap = 0;
    // stage timing: NSTAGE+1 events per timed run, reused across enablements
    std::vector<epic_tile_rule_t> rules;  // relaxation tile by frame size
    bool timing = false;
    std::vector<cudaEvent_t> tev;
    int timed_runs = 0;
    std::string err;
};

static constexpr int NSTAGE = 7;  // prepare .. write-out, pruning

namespace {

const char *status_name(int s) {
    switch (s) {
    case EPIC_OK: return "ok";
    case EPIC_ERR_INVALID: return "invalid input (argument or match outside the image)";
    case EPIC_ERR_OOM: return "out of device memory";
    case EPIC_ERR_CUDA: return "CUDA runtime error";
    case EPIC_ERR_NOT_CONVERGED: return "relaxation did not converge within max_passes";
    case EPIC_ERR_TIMEOUT: return "grid barrier wait timed out";
    case EPIC_ERR_CAPACITY: return "capacity exceeded (edge table, node degree or K-NN frontier)";
    default: return "unknown status";
    }
}

int fail(epic_interp_t *h, int code, const std::string &msg) {
    if (h) h->err = msg;
    return code;
}

int cuda_fail(epic_interp_t *h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(h, EPIC_ERR_OOM, m);
    return fail(h, EPIC_ERR_CUDA, m);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int next_pow2(long long x) {
    long long p = 1;
    while (p < x) p <<= 1;
    return (int)p;
}

// Tile shape for the relaxation of an H x W frame: the first installed rule
// covering the frame, else the configured tile (64 x 32 by default; apron 4
// for the sweep schedules of k_dt.cu, none for the warp tiles of
// k_relax.cu).  With warp_tiles_ok = false (the exact variant's runs, which
// need the capped relaxation of k_dt.cu), a warp-tile choice becomes the
// default k_dt.cu tile.
constexpr int SWEEP_WARP_TILES = 2;

// Tile height when neither the configuration nor a rule gives one: 16 rows
// for warp tiles (what the tile autotuner picks for frames above 64 K
// pixels), 32 for the apron tiles.
int default_tile_h(int sweep) { return sweep == SWEEP_WARP_TILES ? 16 : 32; }

void choose_tiles(const epic_config_t &c, const std::vector<epic_tile_rule_t> &rules, int H,
                  int W, int *tw, int *th, int *ap, int *sweep = nullptr,
                  bool warp_tiles_ok = true) {
    const long long P = (long long)H * W;
    int s = c.sweep;
    bool found = false;
    for (const auto &r : rules) {
        if (P <= r.max_pixels) {
            *tw = r.tile_w;
            *th = r.tile_h;
            *ap = r.apron;
            s = r.sweep;
            found = true;
            break;
        }
    }
    if (!found) {
        *tw = c.tile_w > 0 ? c.tile_w : 64;
        *th = c.tile_h > 0 ? c.tile_h : default_tile_h(s);
        *ap = c.apron >= 0 ? c.apron : (s == SWEEP_WARP_TILES ? 0 : 4);
    }
    if (s == SWEEP_WARP_TILES) {
        if (warp_tiles_ok) {
            *tw = epic::RELAX_TILE_W;
            *th = std::min(*th, epic::RELAX_MAX_ROWS);
            *ap = 0;
        } else {
            *tw = 64;
            *th = 32;
            *ap = 4;
            s = 0;
        }
    }
    if (sweep) *sweep = s;
}

// The interpolator's relaxation kernel for this handle: the warp tiles of
// k_relax.cu when the configuration and every tile rule ask for them, else
// k_dt.cu (a frame whose rule asks for warp tiles then takes the default
// k_dt.cu tile).  A property of the handle, not of a batch, so that a
// captured launch sequence replays for any batch.
bool uses_warp_tiles(const epic_config_t &c, const std::vector<epic_tile_rule_t> &rules) {
    if (c.sweep != SWEEP_WARP_TILES) return false;
    for (const auto &r : rules)
        if (r.sweep != SWEEP_WARP_TILES) return false;
    return true;
}

struct Layout {
    size_t keys, tile_start, tile_fill, tile_seeds, tile_stamp, hkeys, hw, deg, wmin, wmin2, wnear,
        row, adj, models,
        fallback, knn_idx, knn_dist, knn_count, info, keep, pruned, kept_index, end;
};

// K-NN lists hold max(K of the first pass, K of the second) entries per match
int knn_cap(const PairDev &P) { return std::max(P.K, P.K2); }

Layout layout_pair(size_t base, const PairDev &P, int max_degree, bool keep, bool prune) {
    Layout L;
    size_t o = align_up(base, 256);
    const size_t npx = (size_t)P.H * P.W;
    const size_t T = (size_t)P.tiles_x * P.tiles_y;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.keys = take(npx * sizeof(pkey_t));
    L.tile_start = take((T + 1) * sizeof(int));
    L.tile_fill = take(T * sizeof(int));
    L.tile_seeds = take((size_t)P.N * sizeof(int));
    L.tile_stamp = take(T * sizeof(int));
    L.hkeys = take((size_t)P.hash_cap * sizeof(pkey_t));
    L.hw = take((size_t)P.hash_cap * sizeof(unsigned));
    L.deg = take((size_t)P.N * sizeof(int));
    L.wmin = take((size_t)P.N * sizeof(unsigned));
    L.wmin2 = take((size_t)P.N * sizeof(unsigned));
    L.wnear = take((size_t)P.N * sizeof(int));
    L.row = take(((size_t)P.N + 1) * sizeof(int));
    // CSR adjacency: at most one entry per direction of every table slot
    L.adj = take((size_t)P.hash_cap * 2 * sizeof(uint4));
    (void)max_degree;
    L.models = take((size_t)P.N * 2 * sizeof(float4));
    L.fallback = take((size_t)P.N * sizeof(int));
    L.knn_idx = keep ? take((size_t)P.N * knn_cap(P) * sizeof(int)) : 0;
    L.knn_dist = keep ? take((size_t)P.N * knn_cap(P) * sizeof(float)) : 0;
    L.knn_count = keep ? take((size_t)P.N * sizeof(int)) : 0;
    L.info = take(4 * sizeof(int));
    L.keep = prune ? take((size_t)P.N * sizeof(int)) : 0;
    L.pruned = prune ? take((size_t)P.N * sizeof(float4)) : 0;
    L.kept_index = prune ? take((size_t)P.N * sizeof(int)) : 0;
    L.end = o;
    return L;
}

PairDev make_pair_desc(const epic_config_t &c, const std::vector<epic_tile_rule_t> &rules,
                       const epic_pair_desc_t &d) {
    PairDev P{};
    P.C = d.cost_map;
    P.matches = reinterpret_cast<const float4 *>(d.matches);
    P.flow = d.flow_out;
    P.H = d.H;
    P.W = d.W;
    P.N = d.N;
    P.K = std::min(d.K, d.N);
    P.K2 = P.K;
    if (c.prune) {
        // first pass: the NW estimate with prune_K neighbours
        P.K = std::min(c.prune_K, d.N);
    }
    P.a = d.a;
    choose_tiles(c, rules, d.H, d.W, &P.tile_w, &P.tile_h, &P.apron, &P.sweep,
                 uses_warp_tiles(c, rules));
    P.tiles_x = (d.W + P.tile_w - 1) / P.tile_w;
    P.tiles_y = (d.H + P.tile_h - 1) / P.tile_h;
    P.hash_cap = std::max(1024, next_pow2(8LL * d.N));
    P.flow_vec_ok = ((uintptr_t)d.flow_out % 16) == 0;
    return P;
}

// cuTensorMapEncodeTiled, fetched from the driver once through the runtime
// (no link dependency on the driver library); null if unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Tensor maps for TMA staging of the relaxation's cost tiles; leaves
// tma_cost = 0 (plain loads) when a TMA requirement does not hold: a
// 16-byte-aligned base, a row pitch that is a multiple of 16 bytes, and box
// sides of at most 256 elements.
void encode_cost_maps(PairDev &P) {
    P.tma_cost = 0;
    EncodeTiledFn fn = encode_tiled();
    if (!fn || ((uintptr_t)P.C % 16) != 0 || ((size_t)P.W * 4) % 16 != 0) return;
    const int rh_f = P.tile_h + 2 * P.apron + 2, rh_a = P.tile_h + 2;
    const int bw_f = (P.tile_w + 2 * P.apron + 2 + 3 + 3) / 4 * 4;
    const int bw_a = (P.tile_w + 2 + 3 + 3) / 4 * 4;
    if (bw_f > 256 || rh_f > 256 || bw_a > 256 || rh_a > 256) return;
    const cuuint64_t dims[2] = {(cuuint64_t)P.W, (cuuint64_t)P.H};
    const cuuint64_t strides[1] = {(cuuint64_t)P.W * 4};
    const cuuint32_t estr[2] = {1, 1};
    const cuuint32_t box_f[2] = {(cuuint32_t)bw_f, (cuuint32_t)rh_f};
    const cuuint32_t box_a[2] = {(cuuint32_t)bw_a, (cuuint32_t)rh_a};
    void *base = const_cast<float *>(P.C);
    if (fn(&P.tm_cost_fresh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box_f, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        fn(&P.tm_cost_again, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box_a, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return;
    P.tma_bw_fresh = bw_f;
    P.tma_bw_again = bw_a;
    P.tma_cost = 1;
}

// Tensor maps of the warp-tile relaxation (k_relax.cu): the pair's keys as a
// W x H array of 8-byte elements with boxes of 68 x (tile_h + 2), and its
// cost map as float32 with boxes of 72 x (tile_h + 2); both boxes start at
// an x coordinate that is a multiple of 64 minus 2 (keys) or 4 (costs), so
// every copy starts on a 16-byte boundary.  Leaves tma_warp = 0 (plain
// loads) unless both maps can be encoded: 16-byte-aligned bases and row
// pitches that are multiples of 16 bytes (W even for the keys, W a multiple
// of 4 for the costs).
void encode_warp_maps(PairDev &P) {
    P.tma_warp = 0;
    if (P.sweep != SWEEP_WARP_TILES) return;
    EncodeTiledFn fn = encode_tiled();
    if (!fn || ((uintptr_t)P.C % 16) != 0 || ((uintptr_t)P.keys % 16) != 0 ||
        ((size_t)P.W * 4) % 16 != 0 || P.tile_h + 2 > 256)
        return;
    const cuuint64_t dims[2] = {(cuuint64_t)P.W, (cuuint64_t)P.H};
    const cuuint64_t kstr[1] = {(cuuint64_t)P.W * 8};
    const cuuint64_t cstr[1] = {(cuuint64_t)P.W * 4};
    const cuuint32_t estr[2] = {1, 1};
    const cuuint32_t kbox[2] = {68u, (cuuint32_t)(P.tile_h + 2)};
    const cuuint32_t cbox[2] = {72u, (cuuint32_t)(P.tile_h + 2)};
    if (fn(&P.tm_warp_keys, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, P.keys, dims, kstr, kbox, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        fn(&P.tm_warp_cost, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(P.C), dims,
           cstr, cbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return;
    P.tma_warp = 1;
}

int validate(epic_interp_t *h, const epic_pair_desc_t &d, int i) {
    char buf[256];
    if (!d.cost_map || !d.matches || !d.flow_out) {
        snprintf(buf, sizeof buf, "pair %d: null pointer", i);
        return fail(h, EPIC_ERR_INVALID, buf);
    }
    if (d.H < 1 || d.W < 1 || d.N < 1 || d.K < 1 || !(d.a > 0.f) || !std::isfinite(d.a)) {
        snprintf(buf, sizeof buf,
                 "pair %d: need H, W, N, K >= 1 and finite a > 0 (H=%d W=%d N=%d K=%d a=%g)",
                 i, d.H, d.W, d.N, d.K, (double)d.a);
        return fail(h, EPIC_ERR_INVALID, buf);
    }
    if ((long long)d.H * d.W > (1LL << 30) || d.N > epic::MAX_LABELS) {
        snprintf(buf, sizeof buf, "pair %d: frame or match count too large", i);
        return fail(h, EPIC_ERR_INVALID, buf);
    }
    if (((uintptr_t)d.matches % 16) != 0) {
        snprintf(buf, sizeof buf, "pair %d: matches must be 16-byte aligned", i);
        return fail(h, EPIC_ERR_INVALID, buf);
    }
    return EPIC_OK;
}

int wait_last(epic_interp_t *h) {
    cudaError_t e = cudaStreamSynchronize(h->last_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    return EPIC_OK;
}

int ensure_arena(epic_interp_t *h, size_t need) {
    if (need <= h->arena_bytes) return EPIC_OK;
    int rc = wait_last(h);
    if (rc) return rc;
    if (h->arena) cudaFree(h->arena);
    h->arena = nullptr;
    h->arena_bytes = 0;
    size_t sz = align_up(need + need / 4, 1 << 20);
    cudaError_t e = cudaMalloc(&h->arena, sz);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(h, e, "arena cudaMalloc");
    }
    h->arena_bytes = sz;
    return EPIC_OK;
}

void drop_graphs(epic_interp_t *h) {
    for (auto &sl : h->slot) {
        if (sl.graph) cudaGraphExecDestroy(sl.graph);
        sl.graph = nullptr;
    }
}

int ensure_table(epic_interp_t *h, size_t need) {
    if (need <= h->table_cap) return EPIC_OK;
    int rc = wait_last(h);
    if (rc) return rc;
    drop_graphs(h);
    size_t sz = align_up(need * 2, 4096);
    for (auto &sl : h->slot) {
        if (sl.done && sl.pending) cudaEventSynchronize(sl.done);
        sl.pending = false;
        if (sl.dev) cudaFree(sl.dev);
        if (sl.host) cudaFreeHost(sl.host);
        sl.dev = nullptr;
        sl.host = nullptr;
        cudaError_t e = cudaMalloc(&sl.dev, sz);
        if (e != cudaSuccess) { h->table_cap = 0; return cuda_fail(h, e, "table cudaMalloc"); }
        e = cudaMallocHost(&sl.host, sz);
        if (e != cudaSuccess) { h->table_cap = 0; return cuda_fail(h, e, "table cudaMallocHost"); }
    }
    h->table_cap = sz;
    return EPIC_OK;
}

int read_state(epic_interp_t *h) {
    cudaError_t e = cudaMemcpyAsync(h->state_host, h->state, sizeof(RunState),
                                    cudaMemcpyDeviceToHost, h->last_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "state read");
    e = cudaStreamSynchronize(h->last_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    return EPIC_OK;
}

int check_pair(epic_interp_t *h, int pair) {
    if (!h) return EPIC_ERR_INVALID;
    if (pair < 0 || pair >= (int)h->pairs.size())
        return fail(h, EPIC_ERR_INVALID, "pair index out of range of the last run");
    if (!h->pruned) return EPIC_OK;
    // a pruned run rewrote the pair's matches, N and K on the device
    int rc = wait_last(h);
    if (rc) return rc;
    PairDev d;
    cudaError_t e = cudaMemcpy(&d, h->pairs_dev + pair, sizeof d, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "pair descriptor read");
    h->pairs[pair].matches = d.matches;
    h->pairs[pair].N = d.N;
    h->pairs[pair].K = d.K;
    return EPIC_OK;
}

}  // namespace

extern "C" {

void epic_config_default(epic_config_t *c) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->max_H = 436;
    c->max_W = 1024;
    c->max_N = 5000;
    c->max_K = 100;
    c->max_pairs = 1;
    c->max_passes = 4096;
    c->weight_squared = 1;
    c->fallback_eps = 1e-10f;
    c->tile_w = 0;
    c->tile_h = 0;
    c->apron = -1;
    c->keep_intermediates = 0;
    c->max_degree = 32;
    c->use_graphs = 0;
    c->estimator = 0;
    c->prune = 0;
    c->prune_threshold = 5.f;
    c->prune_K = 25;
    c->sweep = SWEEP_WARP_TILES;
}

int epic_interp_create(epic_interp_t **out, int device, const epic_config_t *cfg) {
    if (!out) return EPIC_ERR_INVALID;
    *out = nullptr;
    epic_interp_t *h = new epic_interp_t();
    if (cfg) h->cfg = *cfg; else epic_config_default(&h->cfg);
    epic_config_t &c = h->cfg;
    if (c.max_passes <= 0) c.max_passes = 4096;
    if (c.max_degree <= 0) c.max_degree = 32;
    if (!(c.fallback_eps > 0.f)) c.fallback_eps = 1e-10f;
    if (c.max_pairs <= 0) c.max_pairs = 1;
    if (c.prune_K <= 0) c.prune_K = 25;
    c.max_K = std::min(c.max_K, (int)EPIC_MAX_K);
    if (c.sweep < 0 || c.sweep > SWEEP_WARP_TILES) c.sweep = SWEEP_WARP_TILES;
    if ((c.estimator != 0 && c.estimator != 1) || !(c.prune_threshold >= 0.f) ||
        !std::isfinite(c.prune_threshold)) {
        int r = fail(h, EPIC_ERR_INVALID, "estimator must be 0 or 1, prune_threshold finite >= 0");
        delete h;
        return r;
    }
    // warp tiles are 64 columns (a configured width is ignored) and 1..32 rows
    const bool bad_tile = c.sweep == SWEEP_WARP_TILES
                              ? c.tile_h > epic::RELAX_MAX_ROWS
                              : (c.tile_w > 0 && c.tile_w < 8) || (c.tile_h > 0 && c.tile_h < 8) ||
                                    c.tile_w > 256 || c.tile_h > 256;
    if (bad_tile) {
        int r = fail(h, EPIC_ERR_INVALID,
                     "tile sides must be in [8, 256] (warp tiles: at most 32 rows)");
        delete h;
        return r;
    }
    h->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete h; return EPIC_ERR_CUDA; }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) { delete h; return EPIC_ERR_CUDA; }
    h->num_sms = prop.multiProcessorCount;
    h->smem_optin = (int)prop.sharedMemPerBlockOptin;
    h->smem_per_sm = (int)prop.sharedMemPerMultiprocessor;
    h->smem_reserved = (int)prop.reservedSharedMemPerBlock;
    // the run state, then a scratch counter
    e = cudaMalloc(&h->state, sizeof(RunState) + 64);
    if (e != cudaSuccess) { delete h; return EPIC_ERR_OOM; }
    h->scratch_count = reinterpret_cast<int *>(reinterpret_cast<char *>(h->state) + sizeof(RunState) + 32);
    cudaMemset(h->state, 0, sizeof(RunState) + 64);
    e = cudaMallocHost(&h->state_host, sizeof(RunState));
    if (e != cudaSuccess) { epic_interp_destroy(h); return EPIC_ERR_OOM; }
    for (auto &sl : h->slot) {
        e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e != cudaSuccess) { epic_interp_destroy(h); return EPIC_ERR_CUDA; }
    }
    // size the arena for the configured maxima
    epic_pair_desc_t d{};
    d.cost_map = reinterpret_cast<const float *>(16);
    d.matches = reinterpret_cast<const float *>(16);
    d.flow_out = reinterpret_cast<float *>(16);
    d.H = std::max(1, c.max_H);
    d.W = std::max(1, c.max_W);
    d.N = std::max(1, c.max_N);
    d.K = std::max(1, c.max_K);
    d.a = 1.f;
    PairDev P = make_pair_desc(c, h->rules, d);
    size_t per = layout_pair(0, P, c.max_degree, c.keep_intermediates != 0, c.prune != 0).end;
    // pairs, then the K-NN retry list of the batch (one int per match)
    int rc = ensure_arena(h, per * (size_t)c.max_pairs + 256 +
                                 sizeof(int) * (size_t)d.N * (size_t)c.max_pairs);
    if (rc) { epic_interp_destroy(h); return rc; }
    rc = ensure_table(h, 4096);
    if (rc) { epic_interp_destroy(h); return rc; }
    *out = h;
    return EPIC_OK;
}

int epic_interp_run_batch(epic_interp_t *h, const epic_pair_desc_t *descs, int n,
                          void *stream_) {
    if (!h) return EPIC_ERR_INVALID;
    if (!descs || n < 1) return fail(h, EPIC_ERR_INVALID, "empty batch");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    epic_config_t c = h->cfg;
    if (h->force_keep) {
        c.keep_intermediates = 1;
        c.use_graphs = 0;
        c.prune = 0;
    }
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    for (int i = 0; i < n; ++i) {
        int rc = validate(h, descs[i], i);
        if (rc) return rc;
    }
    // descriptors and arena layout
    std::vector<PairDev> P(n);
    std::vector<Layout> L(n);
    size_t off = 0;
    int max_tw = 8, max_th = 8, max_ap = 0, max_K = 1;
    size_t total_N = 0;
    for (int i = 0; i < n; ++i) {
        P[i] = make_pair_desc(c, h->rules, descs[i]);
        if (P[i].apron + 1 > std::min(P[i].tile_w, P[i].tile_h) || P[i].apron > 64)
            return fail(h, EPIC_ERR_INVALID,
                        "apron must be smaller than the tile sides and at most 64");
        L[i] = layout_pair(off, P[i], c.max_degree, c.keep_intermediates != 0, c.prune != 0);
        off = L[i].end;
        max_tw = std::max(max_tw, P[i].tile_w);
        max_th = std::max(max_th, P[i].tile_h);
        max_ap = std::max(max_ap, P[i].apron);
        max_K = std::max(max_K, knn_cap(P[i]));
        total_N += (size_t)P[i].N;
    }
    // the K-NN retry list: every match of the batch fits, since a match is
    // queued at most once per pass
    const size_t retry_off = align_up(off, 256);
    off = retry_off + sizeof(int) * total_N;
    // the relaxation's work queue and queued flags: one slot each per tile
    size_t total_T = 0;
    for (int i = 0; i < n; ++i) total_T += (size_t)P[i].tiles_x * P[i].tiles_y;
    const size_t rq_off = align_up(off, 256);
    off = rq_off + 2 * sizeof(int) * total_T;
    if (max_K > EPIC_MAX_K)
        return fail(h, EPIC_ERR_INVALID, "K (clamped to N) above EPIC_MAX_K");
    int rc = ensure_arena(h, off);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        encode_cost_maps(P[i]);
        char *b = h->arena;
        P[i].keys = reinterpret_cast<pkey_t *>(b + L[i].keys);
        P[i].tile_start = reinterpret_cast<int *>(b + L[i].tile_start);
        P[i].tile_fill = reinterpret_cast<int *>(b + L[i].tile_fill);
        P[i].tile_seeds = reinterpret_cast<int *>(b + L[i].tile_seeds);
        P[i].tile_stamp = reinterpret_cast<int *>(b + L[i].tile_stamp);
        P[i].hkeys = reinterpret_cast<pkey_t *>(b + L[i].hkeys);
        P[i].hw = reinterpret_cast<unsigned *>(b + L[i].hw);
        P[i].deg = reinterpret_cast<int *>(b + L[i].deg);
        P[i].wmin = reinterpret_cast<unsigned *>(b + L[i].wmin);
        P[i].wmin2 = reinterpret_cast<unsigned *>(b + L[i].wmin2);
        P[i].wnear = reinterpret_cast<int *>(b + L[i].wnear);
        P[i].row = reinterpret_cast<int *>(b + L[i].row);
        P[i].adj = reinterpret_cast<uint4 *>(b + L[i].adj);
        P[i].models = reinterpret_cast<float4 *>(b + L[i].models);
        P[i].fallback = reinterpret_cast<int *>(b + L[i].fallback);
        if (c.keep_intermediates) {
            P[i].knn_idx = reinterpret_cast<int *>(b + L[i].knn_idx);
            P[i].knn_dist = reinterpret_cast<float *>(b + L[i].knn_dist);
            P[i].knn_count = reinterpret_cast<int *>(b + L[i].knn_count);
        }
        P[i].info = reinterpret_cast<int *>(b + L[i].info);
        encode_warp_maps(P[i]);
        if (c.prune) {
            P[i].keep = reinterpret_cast<int *>(b + L[i].keep);
            P[i].pruned = reinterpret_cast<float4 *>(b + L[i].pruned);
            P[i].kept_index = reinterpret_cast<int *>(b + L[i].kept_index);
        }
    }
    // batch table: BatchArgs, PairDev[n], then 5 prefix arrays of n+1 ints
    std::vector<int> tile_base(n + 1), match_base(n + 1), chunk_base(n + 1),
        hash_base(n + 1), clear_base(n + 1);
    long long tt = 0, tm = 0, tc = 0, th = 0, tcl = 0;
    for (int i = 0; i < n; ++i) {
        tile_base[i] = (int)tt;
        match_base[i] = (int)tm;
        chunk_base[i] = (int)tc;
        hash_base[i] = (int)th;
        clear_base[i] = (int)tcl;
        tt += (long long)P[i].tiles_x * P[i].tiles_y;
        tm += P[i].N;
        tc += ((long long)P[i].H * P[i].W + epic::WRITEOUT_CHUNK - 1) / epic::WRITEOUT_CHUNK;
        th += P[i].hash_cap;
        tcl += ((long long)P[i].hash_cap + epic::CLEAR_CHUNK - 1) / epic::CLEAR_CHUNK;
    }
    if (tt > INT32_MAX || tm > INT32_MAX || tc > INT32_MAX || th > INT32_MAX || tcl > INT32_MAX)
        return fail(h, EPIC_ERR_INVALID, "batch too large");
    tile_base[n] = (int)tt;
    match_base[n] = (int)tm;
    chunk_base[n] = (int)tc;
    hash_base[n] = (int)th;
    clear_base[n] = (int)tcl;
    const size_t args_bytes = align_up(sizeof(BatchArgs), 256);
    const size_t pd_bytes = align_up(sizeof(PairDev) * n, 256);
    const size_t pre_bytes = sizeof(int) * (n + 1);
    const size_t pre_stride = align_up(pre_bytes, 256);
    const size_t table_bytes = args_bytes + pd_bytes + 5 * pre_stride;
    rc = ensure_table(h, table_bytes);
    if (rc) return rc;

    // graph replay applies when the launch shapes chosen below do not depend
    // on this batch: kernel sizes from the configured maxima
    // graph launches size the relaxation's shared memory for the largest
    // tile the handle can pick (configured tile or any rule)
    const bool warp_tiles = uses_warp_tiles(c, h->rules);
    // the configured tile counts unless a rule covers every frame size
    bool rules_cover_all = false;
    for (const auto &r : h->rules) rules_cover_all |= r.max_pixels >= (1LL << 30);
    int cfg_tw = c.tile_w > 0 ? c.tile_w : 64,
        cfg_th = c.tile_h > 0 ? c.tile_h : default_tile_h(c.sweep);
    int cfg_ap = c.apron >= 0 ? c.apron : (warp_tiles ? 0 : 4);
    if (rules_cover_all) cfg_tw = cfg_th = 1, cfg_ap = 0;
    for (const auto &r : h->rules) {
        cfg_tw = std::max(cfg_tw, r.tile_w);
        cfg_th = std::max(cfg_th, r.tile_h);
        cfg_ap = std::max(cfg_ap, r.apron);
    }
    if (warp_tiles) {
        cfg_tw = epic::RELAX_TILE_W;
        cfg_th = std::min(cfg_th, epic::RELAX_MAX_ROWS);
        cfg_ap = 0;
    }
    const int cfg_K = std::min((int)EPIC_MAX_K, std::max(c.max_K, c.prune ? c.prune_K : 1));
    const bool graph = c.use_graphs && stream != nullptr && !h->timing && max_K <= cfg_K &&
                       max_tw <= cfg_tw && max_th <= cfg_th && max_ap <= cfg_ap;
    const int knn_K = graph ? cfg_K : max_K;
    const int dt_tw = graph ? cfg_tw : max_tw, dt_th = graph ? cfg_th : max_th;
    const int dt_ap = graph ? cfg_ap : max_ap;

    Handle::Slot &sl = h->slot[h->next_slot];
    h->next_slot ^= 1;
    if (sl.pending) {
        e = cudaEventSynchronize(sl.done);  // the slot's previous run has finished
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
        sl.pending = false;
    }
    BatchArgs a{};
    a.pairs = reinterpret_cast<const PairDev *>(sl.dev + args_bytes);
    auto pre_dev = [&](int k) {
        return reinterpret_cast<const int *>(sl.dev + args_bytes + pd_bytes + k * pre_stride);
    };
    a.npairs = n;
    a.tile_base = pre_dev(0);
    a.match_base = pre_dev(1);
    a.chunk_base = pre_dev(2);
    a.hash_base = pre_dev(3);
    a.clear_base = pre_dev(4);
    a.total_tiles = (int)tt;
    a.total_matches = (int)tm;
    a.total_chunks = (int)tc;
    a.total_hash = (int)th;
    a.total_clear = (int)tcl;
    a.max_degree = c.max_degree;
    const epic::LaunchCfg size_lc{h->num_sms, h->smem_optin, stream, h->smem_per_sm,
                                  h->smem_reserved};
    epic::knn_table_sizes(knn_K, size_lc, &a.knn_hs, &a.knn_fs);
    a.knn_kmax = knn_K;
    a.knn_retry_list = reinterpret_cast<int *>(h->arena + retry_off);
    a.relax_queue = reinterpret_cast<int *>(h->arena + rq_off);
    a.relax_queued = a.relax_queue + total_T;
    a.max_passes = c.max_passes;
    a.weight_squared = c.weight_squared ? 1 : 0;
    a.fallback_eps = c.fallback_eps;
    a.estimator = c.prune ? 1 : c.estimator;
    a.final_estimator = c.estimator;
    a.write_keep = c.prune ? 1 : 0;
    a.prune_threshold = c.prune_threshold;
    a.state = h->state;
    if (epic::knn_warps_per_cta(knn_K, size_lc) < 1)
        return fail(h, EPIC_ERR_INVALID, "K too large for the per-warp search tables");
    if ((warp_tiles ? epic::relax_smem_bytes(dt_th) : epic::dt_smem_bytes(dt_tw, dt_th, dt_ap)) >
        (size_t)h->smem_optin)
        return fail(h, EPIC_ERR_INVALID, "relaxation tile does not fit in shared memory");

    char *hs = sl.host;
    memcpy(hs, &a, sizeof(BatchArgs));
    memcpy(hs + args_bytes, P.data(), sizeof(PairDev) * n);
    const int *pres[5] = {tile_base.data(), match_base.data(), chunk_base.data(),
                          hash_base.data(), clear_base.data()};
    for (int k = 0; k < 5; ++k) memcpy(hs + args_bytes + pd_bytes + k * pre_stride, pres[k], pre_bytes);
    const BatchArgs *dev_a = reinterpret_cast<const BatchArgs *>(sl.dev);

    epic::LaunchCfg lc{h->num_sms, h->smem_optin, stream, h->smem_per_sm, h->smem_reserved};
    BatchArgs *dev_rw = reinterpret_cast<BatchArgs *>(sl.dev);
    auto relax = [&]() -> cudaError_t {
        return warp_tiles ? epic::launch_relax(a, dev_a, lc, dt_th, graph, nullptr)
                          : epic::launch_dt(a, dev_a, lc, dt_tw, dt_th, dt_ap, graph, nullptr);
    };
    const bool prune = c.prune != 0;
    // ev (timing only): a start and an end event per stage
    auto enqueue = [&](cudaEvent_t *ev, size_t copy_bytes) -> cudaError_t {
        auto mark = [&](int i) {
            if (ev) cudaEventRecord(ev[i], stream);
        };
        cudaError_t r = cudaMemcpyAsync(sl.dev, sl.host, copy_bytes, cudaMemcpyHostToDevice, stream);
        if (r) return r;
        mark(12);
        if (prune) {
            // first pass: NW estimate at every match and its keep flag, then
            // the compaction that rewrites the device tables for the second
            if ((r = epic::launch_prepare(a, dev_a, lc))) return r;
            if ((r = relax())) return r;
            if ((r = epic::launch_edges(a, dev_a, lc, dt_tw, dt_th))) return r;
            if ((r = epic::launch_scatter(a, dev_a, lc))) return r;
            if ((r = epic::launch_knn_fit(a, dev_a, lc, knn_K))) return r;
            if ((r = epic::launch_compact(a, dev_rw, lc))) return r;
        }
        mark(13);
        mark(0);
        if ((r = epic::launch_prepare(a, dev_a, lc))) return r;
        mark(1);
        mark(2);
        if ((r = relax())) return r;
        mark(3);
        mark(4);
        if ((r = epic::launch_edges(a, dev_a, lc, dt_tw, dt_th))) return r;
        mark(5);
        mark(6);
        if ((r = epic::launch_scatter(a, dev_a, lc))) return r;
        mark(7);
        mark(8);
        if ((r = epic::launch_knn_fit(a, dev_a, lc, knn_K))) return r;
        mark(9);
        mark(10);
        if ((r = epic::launch_writeout(a, dev_a, lc))) return r;
        mark(11);
        return cudaSuccess;
    };
    if (graph) {
        if (!sl.graph) {
            // capture the whole sequence once; the copy node uploads the
            // slot's entire staging buffer, so any later batch that fits
            // replays the same graph
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t le = enqueue(nullptr, h->table_cap);
                e = cudaStreamEndCapture(stream, &g);
                if (le != cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                sl.graph = nullptr;
                return cuda_fail(h, e, "graph capture");
            }
        }
        e = cudaGraphLaunch(sl.graph, stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
    } else {
        cudaEvent_t *ev = nullptr;
        if (h->timing) {
            size_t need = (size_t)(h->timed_runs + 1) * (2 * NSTAGE);
            while (h->tev.size() < need) {
                cudaEvent_t x;
                if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
                h->tev.push_back(x);
            }
            ev = &h->tev[(size_t)h->timed_runs * (2 * NSTAGE)];
            h->timed_runs++;
        }
        e = enqueue(ev, table_bytes);
        if (e != cudaSuccess) return cuda_fail(h, e, "launch");
    }
    e = cudaEventRecord(sl.done, stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventRecord");
    sl.pending = true;
    h->pairs = P;
    h->pairs_dev = a.pairs;
    h->pruned = prune;
    h->n_submitted.resize(n);
    for (int i = 0; i < n; ++i) h->n_submitted[i] = descs[i].N;
    h->last_stream = stream;
    return EPIC_OK;
}

int epic_interp_run(epic_interp_t *h, const float *cost_map, const float *matches,
                    int H, int W, int N, int K, float a, float *flow_out, void *stream) {
    epic_pair_desc_t d{cost_map, matches, H, W, N, K, a, flow_out};
    return epic_interp_run_batch(h, &d, 1, stream);
}

int epic_interp_run_host(epic_interp_t *h, const float *cost_map, const float *matches,
                         int H, int W, int N, int K, float a, float *flow_out,
                         void *stream_) {
    if (!h) return EPIC_ERR_INVALID;
    if (!cost_map || !matches || !flow_out || H < 1 || W < 1 || N < 1)
        return fail(h, EPIC_ERR_INVALID, "run_host: bad arguments");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    const size_t nC = (size_t)H * W, nM = (size_t)N * 4, nF = (size_t)H * W * 2;
    auto grow = [&](float **p, size_t *cap, size_t need) -> int {
        if (need <= *cap) return EPIC_OK;
        int rc = wait_last(h);
        if (rc) return rc;
        if (*p) cudaFree(*p);
        *p = nullptr;
        *cap = 0;
        cudaError_t ee = cudaMalloc(p, need * sizeof(float));
        if (ee != cudaSuccess) return cuda_fail(h, ee, "run_host cudaMalloc");
        *cap = need;
        return EPIC_OK;
    };
    int rc = grow(&h->io_C, &h->io_C_n, nC);
    if (!rc) rc = grow(&h->io_M, &h->io_M_n, nM);
    if (!rc) rc = grow(&h->io_F, &h->io_F_n, nF);
    if (rc) return rc;
    if ((e = cudaMemcpyAsync(h->io_C, cost_map, nC * 4, cudaMemcpyHostToDevice, stream)) ||
        (e = cudaMemcpyAsync(h->io_M, matches, nM * 4, cudaMemcpyHostToDevice, stream)))
        return cuda_fail(h, e, "run_host upload");
    rc = epic_interp_run(h, h->io_C, h->io_M, H, W, N, K, a, h->io_F, stream_);
    if (rc) return rc;
    if ((e = cudaMemcpyAsync(flow_out, h->io_F, nF * 4, cudaMemcpyDeviceToHost, stream)))
        return cuda_fail(h, e, "run_host download");
    return epic_interp_sync(h);
}

int epic_interp_run_batch_host(epic_interp_t *h, const epic_pair_desc_t *descs, int n,
                               void *stream_) {
    if (!h) return EPIC_ERR_INVALID;
    if (!descs || n < 1) return fail(h, EPIC_ERR_INVALID, "empty batch");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    for (int i = 0; i < n; ++i) {
        int rc = validate(h, descs[i], i);
        if (rc) return rc;
    }
    // one staging buffer: per pair C, matches, flow (256-byte aligned)
    std::vector<size_t> oc(n), om(n), of(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const size_t px = (size_t)descs[i].H * descs[i].W;
        oc[i] = off; off = align_up(off + px * 4, 256);
        om[i] = off; off = align_up(off + (size_t)descs[i].N * 16, 256);
        of[i] = off; off = align_up(off + px * 8, 256);
    }
    if (off > h->io_C_n * 4) {
        int rc = wait_last(h);
        if (rc) return rc;
        if (h->io_C) cudaFree(h->io_C);
        h->io_C = nullptr;
        h->io_C_n = 0;
        e = cudaMalloc(&h->io_C, off);
        if (e != cudaSuccess) return cuda_fail(h, e, "run_batch_host cudaMalloc");
        h->io_C_n = off / 4;
    }
    char *base = reinterpret_cast<char *>(h->io_C);
    std::vector<epic_pair_desc_t> dev(n);
    for (int i = 0; i < n; ++i) {
        const size_t px = (size_t)descs[i].H * descs[i].W;
        if ((e = cudaMemcpyAsync(base + oc[i], descs[i].cost_map, px * 4,
                                 cudaMemcpyHostToDevice, stream)) ||
            (e = cudaMemcpyAsync(base + om[i], descs[i].matches, (size_t)descs[i].N * 16,
                                 cudaMemcpyHostToDevice, stream)))
            return cuda_fail(h, e, "run_batch_host upload");
        dev[i] = descs[i];
        dev[i].cost_map = reinterpret_cast<const float *>(base + oc[i]);
        dev[i].matches = reinterpret_cast<const float *>(base + om[i]);
        dev[i].flow_out = reinterpret_cast<float *>(base + of[i]);
    }
    int rc = epic_interp_run_batch(h, dev.data(), n, stream_);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        const size_t px = (size_t)descs[i].H * descs[i].W;
        if ((e = cudaMemcpyAsync(descs[i].flow_out, base + of[i], px * 8,
                                 cudaMemcpyDeviceToHost, stream)))
            return cuda_fail(h, e, "run_batch_host download");
    }
    return epic_interp_sync(h);
}

int epic_interp_submit_batch_host(epic_interp_t *h, const epic_pair_desc_t *descs, int n) {
    if (!h) return EPIC_ERR_INVALID;
    if (!descs || n < 1) return fail(h, EPIC_ERR_INVALID, "empty batch");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    for (int i = 0; i < n; ++i) {
        int rc = validate(h, descs[i], i);
        if (rc) return rc;
    }
    if (!h->st_up) {
        cudaStream_t *ss[3] = {&h->st_up, &h->st_run, &h->st_down};
        for (cudaStream_t *x : ss)
            if ((e = cudaStreamCreateWithFlags(x, cudaStreamNonBlocking)))
                return cuda_fail(h, e, "cudaStreamCreate");
        for (auto &hs : h->hslot) {
            cudaEvent_t *ev[3] = {&hs.up, &hs.ran, &hs.down};
            for (cudaEvent_t *x : ev)
                if ((e = cudaEventCreateWithFlags(x, cudaEventDisableTiming)))
                    return cuda_fail(h, e, "cudaEventCreate");
        }
    }
    Handle::HostSlot &hs = h->hslot[h->next_hslot];
    h->next_hslot ^= 1;
    if (hs.busy) {
        // the batch two calls back: its downloads (hence its run) are done
        if ((e = cudaEventSynchronize(hs.down))) return cuda_fail(h, e, "cudaEventSynchronize");
        hs.busy = false;
    }
    // staging layout: per pair C, matches, flow (256-byte aligned)
    std::vector<size_t> oc(n), om(n), of(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const size_t px = (size_t)descs[i].H * descs[i].W;
        oc[i] = off; off = align_up(off + px * 4, 256);
        om[i] = off; off = align_up(off + (size_t)descs[i].N * 16, 256);
        of[i] = off; off = align_up(off + px * 8, 256);
    }
    if (off > hs.cap) {
        // nothing in flight reads this slot any more
        if (hs.buf) cudaFree(hs.buf);
        hs.buf = nullptr;
        hs.cap = 0;
        if ((e = cudaMalloc(&hs.buf, off))) return cuda_fail(h, e, "submit_batch_host cudaMalloc");
        hs.cap = off;
    }
    std::vector<epic_pair_desc_t> dev(n);
    for (int i = 0; i < n; ++i) {
        const size_t px = (size_t)descs[i].H * descs[i].W;
        if ((e = cudaMemcpyAsync(hs.buf + oc[i], descs[i].cost_map, px * 4,
                                 cudaMemcpyHostToDevice, h->st_up)) ||
            (e = cudaMemcpyAsync(hs.buf + om[i], descs[i].matches, (size_t)descs[i].N * 16,
                                 cudaMemcpyHostToDevice, h->st_up)))
            return cuda_fail(h, e, "submit_batch_host upload");
        dev[i] = descs[i];
        dev[i].cost_map = reinterpret_cast<const float *>(hs.buf + oc[i]);
        dev[i].matches = reinterpret_cast<const float *>(hs.buf + om[i]);
        dev[i].flow_out = reinterpret_cast<float *>(hs.buf + of[i]);
    }
    if ((e = cudaEventRecord(hs.up, h->st_up)) || (e = cudaStreamWaitEvent(h->st_run, hs.up, 0)))
        return cuda_fail(h, e, "submit_batch_host upload event");
    int rc = epic_interp_run_batch(h, dev.data(), n, h->st_run);
    if (rc) return rc;
    if ((e = cudaEventRecord(hs.ran, h->st_run)) ||
        (e = cudaStreamWaitEvent(h->st_down, hs.ran, 0)))
        return cuda_fail(h, e, "submit_batch_host run event");
    for (int i = 0; i < n; ++i) {
        const size_t px = (size_t)descs[i].H * descs[i].W;
        if ((e = cudaMemcpyAsync(descs[i].flow_out, hs.buf + of[i], px * 8,
                                 cudaMemcpyDeviceToHost, h->st_down)))
            return cuda_fail(h, e, "submit_batch_host download");
    }
    if ((e = cudaEventRecord(hs.down, h->st_down))) return cuda_fail(h, e, "submit_batch_host");
    hs.busy = true;
    return EPIC_OK;
}

int epic_interp_sync(epic_interp_t *h) {
    if (!h) return EPIC_ERR_INVALID;
    for (auto &hs : h->hslot) {
        if (!hs.busy) continue;
        cudaError_t e = cudaEventSynchronize(hs.down);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
        hs.busy = false;
    }
    int rc = read_state(h);
    if (rc) return rc;
    int s = h->state_host->status;
    if (s != 0) {
        cudaMemsetAsync(&h->state->status, 0, sizeof(int), h->last_stream);
        cudaStreamSynchronize(h->last_stream);
        return fail(h, s, status_name(s));
    }
    return EPIC_OK;
}

int epic_interp_get_labels(epic_interp_t *h, int pair, int *labels, float *dist,
                           void *stream) {
    int rc = check_pair(h, pair);
    if (rc) return rc;
    cudaError_t e = epic::launch_split_keys(&h->pairs[pair], h->pairs_dev + pair, labels, dist,
                                            reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EPIC_OK : cuda_fail(h, e, "get_labels");
}

int epic_interp_get_edge_count(epic_interp_t *h, int pair, int *n_edges) {
    int rc = check_pair(h, pair);
    if (rc) return rc;
    if (!n_edges) return fail(h, EPIC_ERR_INVALID, "null output");
    rc = wait_last(h);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(n_edges, h->pairs[pair].info, sizeof(int), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? EPIC_OK : cuda_fail(h, e, "get_edge_count");
}

int epic_interp_get_graph(epic_interp_t *h, int pair, int *em, int *en, float *ew,
                          int cap, int *n_edges) {
    int rc = check_pair(h, pair);
    if (rc) return rc;
    if (!em || !en || !ew || !n_edges || cap < 0) return fail(h, EPIC_ERR_INVALID, "null output");
    cudaError_t e = epic::launch_collect_edges(&h->pairs[pair], em, en, ew, cap,
                                               h->scratch_count, h->last_stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->state_host, h->scratch_count, sizeof(int),
                            cudaMemcpyDeviceToHost, h->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->last_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_graph");
    *n_edges = *reinterpret_cast<int *>(h->state_host);
    return *n_edges <= cap ? EPIC_OK : fail(h, EPIC_ERR_CAPACITY, "edge buffer too small");
}

int epic_interp_get_knn(epic_interp_t *h, int pair, int *idx, float *dist, int *count,
                        void *stream_) {
    int rc = check_pair(h, pair);
    if (rc) return rc;
    const PairDev &P = h->pairs[pair];
    if (!P.knn_idx) return fail(h, EPIC_ERR_INVALID, "K-NN lists need keep_intermediates = 1");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    size_t nk = (size_t)P.N * P.K;
    cudaError_t e = cudaSuccess;
    if (idx) e = cudaMemcpyAsync(idx, P.knn_idx, nk * 4, cudaMemcpyDeviceToDevice, s);
    if (!e && dist) e = cudaMemcpyAsync(dist, P.knn_dist, nk * 4, cudaMemcpyDeviceToDevice, s);
    if (!e && count) e = cudaMemcpyAsync(count, P.knn_count, (size_t)P.N * 4, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? EPIC_OK : cuda_fail(h, e, "get_knn");
}

int epic_interp_get_models(epic_interp_t *h, int pair, float *models, int *fallback,
                           void *stream_) {
    int rc = check_pair(h, pair);
    if (rc) return rc;
    const PairDev &P = h->pairs[pair];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    cudaError_t e = cudaSuccess;
    if (models)
        e = cudaMemcpyAsync(models, P.models, (size_t)P.N * 32, cudaMemcpyDeviceToDevice, s);
    if (!e && fallback)
        e = cudaMemcpyAsync(fallback, P.fallback, (size_t)P.N * 4, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? EPIC_OK : cuda_fail(h, e, "get_models");
}

int epic_interp_get_pruning(epic_interp_t *h, int pair, int *keep, int *kept_index,
                            int *n_kept) {
    int rc = check_pair(h, pair);
    if (rc) return rc;
    if (!h->pruned) return fail(h, EPIC_ERR_INVALID, "the last run did not prune (prune = 0)");
    const PairDev &P = h->pairs[pair];
    cudaError_t e = cudaSuccess;
    if (keep)
        e = cudaMemcpy(keep, P.keep, (size_t)h->n_submitted[pair] * sizeof(int),
                       cudaMemcpyDeviceToDevice);
    if (!e && kept_index)
        e = cudaMemcpy(kept_index, P.kept_index, (size_t)P.N * sizeof(int),
                       cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_pruning");
    if (n_kept) *n_kept = P.N;
    return EPIC_OK;
}

int epic_interp_get_passes(epic_interp_t *h, int *passes) {
    if (!h || !passes) return EPIC_ERR_INVALID;
    int rc = read_state(h);
    if (rc) return rc;
    *passes = h->state_host->passes;
    return EPIC_OK;
}

int epic_interp_get_distance_unit(epic_interp_t *h, int pair, int *shift) {
    if (!h || !shift) return EPIC_ERR_INVALID;
    int rc = check_pair(h, pair);
    if (rc) return rc;
    rc = wait_last(h);
    if (rc) return rc;
    PairDev d;
    cudaError_t e = cudaMemcpy(&d, h->pairs_dev + pair, sizeof d, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "pair descriptor read");
    *shift = d.sweep == SWEEP_WARP_TILES
                 ? epic::unit_shift_of(d.cmax_bits, d.seed_reach, d.tile_w, d.tile_h)
                 : 0;
    return EPIC_OK;
}

int epic_interp_get_knn_retries(epic_interp_t *h, int *retries) {
    if (!h || !retries) return EPIC_ERR_INVALID;
    int rc = read_state(h);
    if (rc) return rc;
    *retries = (int)h->state_host->knn_overflow;
    return EPIC_OK;
}

int epic_interp_set_tile_rules(epic_interp_t *h, const epic_tile_rule_t *rules, int n) {
    if (!h) return EPIC_ERR_INVALID;
    if (n < 0 || (n > 0 && !rules)) return fail(h, EPIC_ERR_INVALID, "bad rule list");
    std::vector<epic_tile_rule_t> v(rules, rules + n);
    for (const auto &r : v) {
        if (r.sweep == SWEEP_WARP_TILES) {
            if (r.tile_w != epic::RELAX_TILE_W || r.tile_h < 1 || r.tile_h > epic::RELAX_MAX_ROWS ||
                r.apron != 0 || r.max_pixels < 1)
                return fail(h, EPIC_ERR_INVALID, "warp-tile rule needs 64 x (1..32) tiles, apron 0");
            continue;
        }
        if (r.tile_w < 8 || r.tile_h < 8 || r.tile_w > 256 || r.tile_h > 256 || r.apron < 0 ||
            r.apron > 64 || r.apron + 1 > std::min(r.tile_w, r.tile_h) || r.max_pixels < 1 ||
            (r.sweep != 0 && r.sweep != 1))
            return fail(h, EPIC_ERR_INVALID, "tile rule out of range");
        if (epic::dt_smem_bytes(r.tile_w, r.tile_h, r.apron) > (size_t)h->smem_optin)
            return fail(h, EPIC_ERR_INVALID, "tile rule does not fit in shared memory");
    }
    // graphs were captured for the old maximum tile
    int rc = wait_last(h);
    if (rc) return rc;
    drop_graphs(h);
    h->rules = v;
    return EPIC_OK;
}

int epic_interp_enable_stage_timing(epic_interp_t *h, int enable) {
    if (!h) return EPIC_ERR_INVALID;
    if (h->timed_runs > 0) {
        int rc = wait_last(h);
        if (rc) return rc;
    }
    h->timing = enable != 0;
    h->timed_runs = 0;
    return EPIC_OK;
}

int epic_interp_get_stage_times(epic_interp_t *h, float *ms_out, int n_stages, int *n_runs) {
    if (!h || !ms_out || n_stages < 0 || n_stages > NSTAGE) return EPIC_ERR_INVALID;
    for (int s = 0; s < n_stages; ++s) ms_out[s] = 0.f;
    if (n_runs) *n_runs = h->timed_runs;
    if (h->timed_runs == 0) return EPIC_OK;
    // the write-out's end event (index 11) is the last one a run records
    cudaError_t e = cudaEventSynchronize(h->tev[(size_t)(h->timed_runs - 1) * (2 * NSTAGE) + 11]);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
    for (int r = 0; r < h->timed_runs; ++r) {
        const cudaEvent_t *ev = &h->tev[(size_t)r * (2 * NSTAGE)];
        for (int s = 0; s < n_stages; ++s) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[2 * s], ev[2 * s + 1]);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventElapsedTime");
            ms_out[s] += ms;
        }
    }
    return EPIC_OK;
}

int epic_exact_interp(epic_interp_t *h, const float *cost_map, const float *matches, int H,
                      int W, int N, int K, float a, int metric, float *flow_out,
                      int *knn_idx_out, float *knn_dist_out, void *stream_) {
    if (!h) return EPIC_ERR_INVALID;
    epic_pair_desc_t d{cost_map, matches, H, W, N, K, a, flow_out};
    int rc = validate(h, d, 0);
    if (rc) return rc;
    if (metric != 0 && metric != 1) return fail(h, EPIC_ERR_INVALID, "metric must be 0 or 1");
    if (knn_idx_out && !knn_dist_out)
        return fail(h, EPIC_ERR_INVALID, "knn_idx_out needs knn_dist_out");
    const epic_config_t &c = h->cfg;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    K = std::min(K, N);
    if (epic::exact_smem_bytes(K) > (size_t)h->smem_optin)
        return fail(h, EPIC_ERR_INVALID, "K too large for the per-pixel lists");
    const long long P = (long long)H * W;
    float *D = nullptr;
    if (metric == 0) {
        // single-source relaxations, Cm matches at a time, each a pseudo-pair
        // with one seed; their distances become row m of D [N][P]
        int tw, th, ap, sw;
        choose_tiles(c, h->rules, H, W, &tw, &th, &ap, &sw, false);
        const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th, T = tx * ty;
        const long long chunk_bytes = c.exact_chunk_bytes > 0 ? c.exact_chunk_bytes : (1LL << 30);
        const long long Cm = std::max(1LL, std::min((long long)N, chunk_bytes / (P * 8)));
        const size_t small_ints = (size_t)(T + 1) + T + 1 + T + 1 + 1 + 4;  // per pseudo-pair
        const size_t d_bytes = align_up((size_t)N * P * sizeof(float), 256);
        const size_t k_bytes = align_up((size_t)Cm * P * sizeof(pkey_t), 256);
        const size_t s_bytes = align_up((size_t)Cm * small_ints * sizeof(int), 256);
        const size_t args_bytes = align_up(sizeof(BatchArgs), 256);
        const size_t pd_bytes = align_up(sizeof(PairDev) * Cm, 256);
        const size_t pre_stride = align_up(sizeof(int) * (Cm + 1), 256);
        const size_t t_bytes = args_bytes + pd_bytes + 5 * pre_stride;
        // cap map: its keys, the bins and per-match scratch of its
        // relaxation, the seed offsets, and the approximate run's flow
        const size_t v_ints = (size_t)(T + 1) + T + N + T + N + N + 4;
        const size_t c_bytes = align_up((size_t)P * sizeof(pkey_t), 256) +
                               align_up(v_ints * sizeof(int), 256) +
                               align_up((size_t)N * sizeof(unsigned long long), 256) +
                               align_up((size_t)P * 2 * sizeof(float), 256);
        // worklists of the chunked passes: three lists and the queued marks
        const size_t w_bytes = align_up((size_t)4 * Cm * T * sizeof(int), 256);
        const size_t need = d_bytes + k_bytes + s_bytes + align_up(t_bytes, 256) + c_bytes + w_bytes;
        if (need > h->ex_cap) {
            if ((e = cudaStreamSynchronize(stream)) != cudaSuccess)
                return cuda_fail(h, e, "cudaStreamSynchronize");
            if (h->ex_buf) cudaFree(h->ex_buf);
            h->ex_buf = nullptr;
            h->ex_cap = 0;
            e = cudaMalloc(&h->ex_buf, need);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return cuda_fail(h, e, "exact-variant cudaMalloc");
            }
            h->ex_cap = need;
        }
        char *b = h->ex_buf;
        D = reinterpret_cast<float *>(b);
        pkey_t *keys = reinterpret_cast<pkey_t *>(b + d_bytes);
        int *small = reinterpret_cast<int *>(b + d_bytes + k_bytes);
        char *tdev = b + d_bytes + k_bytes + s_bytes;
        char *cb = tdev + align_up(t_bytes, 256);
        pkey_t *vkeys = reinterpret_cast<pkey_t *>(cb);
        int *vs = reinterpret_cast<int *>(cb + align_up((size_t)P * sizeof(pkey_t), 256));
        unsigned long long *vinit = reinterpret_cast<unsigned long long *>(
            reinterpret_cast<char *>(vs) + align_up(v_ints * sizeof(int), 256));
        float *aflow = reinterpret_cast<float *>(
            reinterpret_cast<char *>(vinit) + align_up((size_t)N * sizeof(unsigned long long), 256));
        int *wl = reinterpret_cast<int *>(cb + c_bytes);   // [3][Cm * T], then [Cm * T] marks
        std::vector<char> thost(t_bytes);
        epic::LaunchCfg lc{h->num_sms, h->smem_optin, stream, h->smem_per_sm, h->smem_reserved};

        // Cap map.  An approximate run keeps its K-NN lists: each match's
        // K-th nearest graph distance bounds its K-th nearest geodesic
        // distance.  A multi-source relaxation seeded with those bounds gives
        // V(p) = min over m of (d(p, m) + bound(m)) >= the K-th nearest
        // distance of p, and V is 1-Lipschitz in the relaxation's metric.
        // The single-source runs below write back only distances within V,
        // so each stops spreading about where its seed stops mattering.
        {
            h->force_keep = true;
            epic_pair_desc_t ad{cost_map, matches, H, W, N, K, a, aflow};
            const int rca = epic_interp_run_batch(h, &ad, 1, stream_);
            h->force_keep = false;
            if (rca) return rca;
            const PairDev &Pa = h->pairs[0];
            if ((e = epic::launch_cap_seed(Pa.knn_dist, Pa.knn_count, N, K, Pa.K, vinit, stream)))
                return cuda_fail(h, e, "exact-variant cap seeds");
            PairDev v{};
            v.C = cost_map;
            v.matches = reinterpret_cast<const float4 *>(matches);
            v.H = H;
            v.W = W;
            v.N = N;
            v.K = 1;
            v.a = 1.f;
            v.tile_w = tw;
            v.tile_h = th;
            v.apron = ap;
            v.sweep = sw;
            v.tiles_x = tx;
            v.tiles_y = ty;
            v.keys = vkeys;
            v.tile_start = vs;
            v.tile_fill = vs + T + 1;
            v.tile_seeds = vs + 2 * T + 1;
            v.tile_stamp = vs + 2 * T + 1 + N;
            v.deg = vs + 3 * T + 1 + N;
            v.wmin = reinterpret_cast<unsigned *>(vs + 3 * T + 1 + 2 * N);
            v.info = vs + 3 * T + 1 + 3 * N;
            v.seed_init = vinit;
            std::vector<int> pre(5 * 2, 0);
            pre[1] = T;          // tiles
            pre[2 + 1] = N;      // matches
            BatchArgs vb{};
            vb.pairs = reinterpret_cast<const PairDev *>(tdev + args_bytes);
            vb.npairs = 1;
            auto vpre = [&](int k) {
                return reinterpret_cast<const int *>(tdev + args_bytes + pd_bytes + k * pre_stride);
            };
            vb.tile_base = vpre(0);
            vb.match_base = vpre(1);
            vb.chunk_base = vpre(2);
            vb.hash_base = vpre(3);
            vb.clear_base = vpre(4);
            vb.total_tiles = T;
            vb.total_matches = N;
            vb.max_degree = 1;
            vb.max_passes = c.max_passes;
            vb.weight_squared = 1;
            vb.fallback_eps = c.fallback_eps;
            vb.state = h->state;
            memcpy(thost.data(), &vb, sizeof vb);
            memcpy(thost.data() + args_bytes, &v, sizeof(PairDev));
            for (int k = 0; k < 5; ++k)
                memcpy(thost.data() + args_bytes + pd_bytes + k * pre_stride, pre.data() + k * 2,
                       sizeof(int) * 2);
            const BatchArgs *dev_v = reinterpret_cast<const BatchArgs *>(tdev);
            if ((e = cudaMemcpyAsync(tdev, thost.data(), t_bytes, cudaMemcpyHostToDevice, stream)) ||
                (e = epic::launch_prepare(vb, dev_v, lc)) ||
                (e = epic::launch_dt(vb, dev_v, lc, tw, th, ap, false, nullptr)) ||
                (e = cudaStreamSynchronize(stream)))
                return cuda_fail(h, e, "exact-variant cap map");
        }
        for (long long m0 = 0; m0 < N; m0 += Cm) {
            const int n = (int)std::min(Cm, (long long)N - m0);
            std::vector<PairDev> pd(n);
            for (int j = 0; j < n; ++j) {
                PairDev &q = pd[j];
                q = PairDev{};
                q.C = cost_map;
                q.matches = reinterpret_cast<const float4 *>(matches) + m0 + j;
                q.H = H;
                q.W = W;
                q.N = 1;
                q.K = 1;
                q.a = 1.f;
                q.tile_w = tw;
                q.tile_h = th;
                q.apron = ap;
                q.sweep = sw;
                q.tiles_x = tx;
                q.tiles_y = ty;
                q.keys = keys + (size_t)j * P;
                int *sp = small + (size_t)j * small_ints;
                q.tile_start = sp;
                q.tile_fill = sp + T + 1;
                q.tile_seeds = sp + 2 * T + 1;
                q.tile_stamp = sp + 2 * T + 2;
                q.deg = sp + 3 * T + 2;
                q.wmin = reinterpret_cast<unsigned *>(sp + 3 * T + 3);
                q.info = sp + 3 * T + 4;
                q.cap = vkeys;
            }
            std::vector<int> pre(5 * (n + 1), 0);
            for (int j = 0; j <= n; ++j) {
                pre[j] = j * T;                 // tiles
                pre[(n + 1) + j] = j;           // matches
            }
            BatchArgs ba{};
            ba.pairs = reinterpret_cast<const PairDev *>(tdev + args_bytes);
            ba.npairs = n;
            auto pre_dev = [&](int k) {
                return reinterpret_cast<const int *>(tdev + args_bytes + pd_bytes + k * pre_stride);
            };
            ba.tile_base = pre_dev(0);
            ba.match_base = pre_dev(1);
            ba.chunk_base = pre_dev(2);
            ba.hash_base = pre_dev(3);
            ba.clear_base = pre_dev(4);
            ba.total_tiles = n * T;
            ba.total_matches = n;
            ba.uniform_tiles = T;
            ba.wl = wl;
            ba.wl_queued = wl + (size_t)3 * n * T;
            ba.max_degree = 1;
            ba.max_passes = c.max_passes;
            ba.weight_squared = 1;
            ba.fallback_eps = c.fallback_eps;
            ba.state = h->state;
            memcpy(thost.data(), &ba, sizeof ba);
            memcpy(thost.data() + args_bytes, pd.data(), sizeof(PairDev) * n);
            for (int k = 0; k < 5; ++k)
                memcpy(thost.data() + args_bytes + pd_bytes + k * pre_stride, pre.data() + k * (n + 1),
                       sizeof(int) * (n + 1));
            const BatchArgs *dev_a = reinterpret_cast<const BatchArgs *>(tdev);
            if ((e = cudaMemcpyAsync(tdev, thost.data(), t_bytes, cudaMemcpyHostToDevice, stream)) ||
                (e = cudaMemsetAsync(ba.wl_queued, 0, sizeof(int) * (size_t)n * T, stream)) ||
                (e = epic::launch_prepare(ba, dev_a, lc)) ||
                (e = epic::launch_dt(ba, dev_a, lc, tw, th, ap, false, nullptr, true)) ||
                (e = epic::launch_keys_to_dist(keys, (long long)n * P, D + m0 * P, stream)) ||
                (e = cudaStreamSynchronize(stream)))
                return cuda_fail(h, e, "exact-variant relaxation");
        }
    }
    epic::ExactArgs x{};
    x.D = D;
    x.matches = reinterpret_cast<const float4 *>(matches);
    x.flow = flow_out;
    x.knn_idx = knn_idx_out;
    x.knn_dist = knn_idx_out ? knn_dist_out : nullptr;
    x.H = H;
    x.W = W;
    x.N = N;
    x.K = K;
    x.a = a;
    x.fallback_eps = c.fallback_eps;
    x.weight_squared = c.weight_squared ? 1 : 0;
    x.estimator = c.estimator;
    if ((e = epic::launch_exact_fit(x, stream)) != cudaSuccess)
        return cuda_fail(h, e, "exact-variant fit");
    h->last_stream = stream;
    return epic_interp_sync(h);
}

int epic_selftest_wait_timeout(epic_interp_t *h, int which, int limit_ms) {
    if (!h || (which != 0 && which != 1) || limit_ms < 1 || limit_ms > 10000)
        return EPIC_ERR_INVALID;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    cudaStream_t s = h->last_stream;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(h, e, "sync");
    if ((e = cudaMemsetAsync(h->state, 0, sizeof(RunState), s)) != cudaSuccess ||
        (e = epic::launch_wait_selftest(h->state, which, (unsigned long long)limit_ms * 1000000ull,
                                        s)) != cudaSuccess)
        return cuda_fail(h, e, "wait self-test");
    return epic_interp_sync(h);   // the recorded status (then cleared)
}

void epic_refine_params_default(epic_refine_params_t *p) {
    if (!p) return;
    p->alpha0 = 1.f;
    p->gamma = 0.7f;
    p->kappa = 5.f;
    p->eps = 1e-3f;
    p->zeta = 0.1f;
    p->omega = 1.6f;
    p->iterations = 5;
    p->sor_iterations = 30;
}

int epic_refine(epic_interp_t *h, const float *I1, const float *I2, int H, int W, int channels,
                float *flow, const epic_refine_params_t *params, void *stream_) {
    if (!h) return EPIC_ERR_INVALID;
    epic_refine_params_t prm;
    if (params) prm = *params; else epic_refine_params_default(&prm);
    if (!I1 || !I2 || !flow || H < 1 || W < 1 || channels < 1 || channels > 4)
        return fail(h, EPIC_ERR_INVALID, "refine: bad arguments");
    if (((uintptr_t)flow % 8) != 0)
        return fail(h, EPIC_ERR_INVALID, "refine: flow must be 8-byte aligned");
    if (!(prm.alpha0 >= 0.f) || !(prm.gamma >= 0.f) || !(prm.kappa >= 0.f) || !(prm.eps > 0.f) ||
        !(prm.zeta > 0.f) || !(prm.omega > 0.f && prm.omega < 2.f) || prm.iterations < 0 ||
        prm.sor_iterations < 0)
        return fail(h, EPIC_ERR_INVALID, "refine: parameter out of range");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    const size_t need = epic::refine_scratch_bytes(H, W, channels);
    if (need > h->rf_cap) {
        if ((e = cudaStreamSynchronize(stream)) != cudaSuccess)
            return cuda_fail(h, e, "cudaStreamSynchronize");
        if (h->rf_buf) cudaFree(h->rf_buf);
        h->rf_buf = nullptr;
        h->rf_cap = 0;
        if ((e = cudaMalloc(&h->rf_buf, need)) != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(h, e, "refine cudaMalloc");
        }
        h->rf_cap = need;
    }
    epic::RefineArgs r{prm.alpha0, prm.gamma, prm.kappa, prm.eps, prm.zeta, prm.omega,
                       prm.iterations, prm.sor_iterations};
    e = epic::launch_refine(I1, I2, H, W, channels, flow, r, h->rf_buf, h->num_sms, stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "refine launch");
    h->last_stream = stream;
    return EPIC_OK;
}

int epic_gradient_cost(const float *image, int frames, int H, int W, int channels,
                       float floor_, float *cost_out, void *stream) {
    if (!image || !cost_out || frames < 1 || H < 1 || W < 1 ||
        (channels != 1 && channels != 3 && channels != 4) || !(floor_ >= 0.f) ||
        !std::isfinite(floor_))
        return EPIC_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return EPIC_ERR_CUDA;
    cudaError_t e = epic::launch_gradcost(image, frames, H, W, channels, floor_, cost_out, sms,
                                          reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

int epic_interp_request_bytes(const epic_interp_t *h, const epic_config_t *cfg, int H, int W,
                              int N, int K, long long *bytes) {
    if (!bytes || H < 1 || W < 1 || N < 1 || K < 1 || N > epic::MAX_LABELS ||
        (long long)H * W > (1LL << 30))
        return EPIC_ERR_INVALID;
    epic_config_t c;
    if (h) c = h->cfg;
    else if (cfg) c = *cfg;
    else epic_config_default(&c);
    static const std::vector<epic_tile_rule_t> no_rules;
    epic_pair_desc_t d{};
    d.cost_map = reinterpret_cast<const float *>(16);
    d.matches = reinterpret_cast<const float *>(16);
    d.flow_out = reinterpret_cast<float *>(16);
    d.H = H;
    d.W = W;
    d.N = N;
    d.K = K;
    d.a = 1.f;
    const PairDev P = make_pair_desc(c, h ? h->rules : no_rules, d);
    // the pair's arena regions (each 256-byte aligned, so a pair placed after
    // any other needs at most its aligned size), its K-NN retry-list slots
    // and its tiles' slots in the relaxation's work queue and queued flags
    const size_t per = layout_pair(0, P, c.max_degree, c.keep_intermediates != 0,
                                   c.prune != 0).end;
    *bytes = (long long)(per + sizeof(int) * (size_t)N +
                         2 * sizeof(int) * (size_t)P.tiles_x * P.tiles_y);
    return EPIC_OK;
}

int epic_interp_launches_per_run(epic_interp_t *h, int n) {
    (void)n;
    // prepare, relaxation, edges, CSR offsets, scatter, the two lightest
    // edges per node, the per-entry bound edge, K-NN + fit and its retry
    // pass, write-out; pruning adds the first pass's nine and the compaction
    return h && h->cfg.prune ? 20 : 10;
}

const char *epic_interp_last_error(epic_interp_t *h) {
    if (!h) return "null handle";
    return h->err.c_str();
}

void epic_interp_destroy(epic_interp_t *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    if (h->arena) cudaFree(h->arena);
    if (h->state) cudaFree(h->state);
    if (h->state_host) cudaFreeHost(h->state_host);
    drop_graphs(h);
    for (auto &sl : h->slot) {
        if (sl.dev) cudaFree(sl.dev);
        if (sl.host) cudaFreeHost(sl.host);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    for (auto &hs : h->hslot) {
        if (hs.buf) cudaFree(hs.buf);
        for (cudaEvent_t x : {hs.up, hs.ran, hs.down})
            if (x) cudaEventDestroy(x);
    }
    for (cudaStream_t x : {h->st_up, h->st_run, h->st_down})
        if (x) cudaStreamDestroy(x);
    if (h->io_C) cudaFree(h->io_C);
    if (h->io_M) cudaFree(h->io_M);
    if (h->io_F) cudaFree(h->io_F);
    if (h->ex_buf) cudaFree(h->ex_buf);
    if (h->rf_buf) cudaFree(h->rf_buf);
    for (cudaEvent_t x : h->tev) cudaEventDestroy(x);
    delete h;
}

}  // extern "C"
