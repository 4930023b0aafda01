// Geodesic assignment map (stage a) without any device allocation.
//
// Some callers cannot let a library allocate device memory: a host
// framework that owns every device allocation and only lends buffers to its
// plugins, or a latency-critical loop in which cudaMalloc's implicit device
// synchronisation and unpredictable latency are not acceptable.  This entry
// point serves them.  It runs the same seed-binning and relaxation kernels as
// epic_interp_run, but their scratch (packed (D, L) keys, seed bins, the run
// state and the grid barrier) lives in one file-scope device array below, so
// the call allocates nothing; the caller provides only inputs and outputs.
//
// The array is part of the library image: every GPU that loads the library
// holds it (about 5 MB) until the process exits.  Its device address belongs
// to the CUDA context that loaded the library's device code, so every call
// looks it up again (cudaGetSymbolAddress, a host-side query) in the context
// current at the call: an address kept from an earlier call would be stale
// after cudaDeviceReset or in another context on the same device.  All
// calls share the array, so calls that overlap on the GPU (from several
// host threads or streams) race; each call clears what must start at zero
// and waits for its own work before returning.
#include <cuda_runtime.h>

#include "epic_internal.cuh"

namespace {

using epic::pkey_t;

constexpr int NA_MAX_PIXELS = 1 << 19;   // e.g. 1024 x 512
constexpr int NA_MAX_MATCHES = 1 << 15;
constexpr int NA_MAX_TILES = 1 << 14;
constexpr int NA_TILE_W = 64, NA_TILE_H = 32, NA_APRON = 4;

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_KEYS = 0;
constexpr size_t OFF_TSTART = align256(OFF_KEYS + sizeof(pkey_t) * NA_MAX_PIXELS);
constexpr size_t OFF_TFILL = align256(OFF_TSTART + sizeof(int) * (NA_MAX_TILES + 1));
constexpr size_t OFF_TSEEDS = align256(OFF_TFILL + sizeof(int) * NA_MAX_TILES);
constexpr size_t OFF_TSTAMP = align256(OFF_TSEEDS + sizeof(int) * NA_MAX_MATCHES);
constexpr size_t OFF_DEG = align256(OFF_TSTAMP + sizeof(int) * NA_MAX_TILES);
constexpr size_t OFF_WMIN = align256(OFF_DEG + sizeof(int) * NA_MAX_MATCHES);
constexpr size_t OFF_INFO = align256(OFF_WMIN + sizeof(unsigned) * NA_MAX_MATCHES);
constexpr size_t OFF_STATE = align256(OFF_INFO + 4 * sizeof(int));
constexpr size_t OFF_PAIR = align256(OFF_STATE + sizeof(epic::RunState));
constexpr size_t OFF_PREFIX = align256(OFF_PAIR + sizeof(epic::PairDev));
constexpr size_t OFF_ARGS = align256(OFF_PREFIX + 5 * 2 * sizeof(int));
constexpr size_t NA_SCRATCH_BYTES = align256(OFF_ARGS + sizeof(epic::BatchArgs));

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

// Device address of the scratch array in the current context, looked up on
// every call (the context may have been reset or replaced since the last).
int scratch_address(unsigned char **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return EPIC_ERR_CUDA;
    *out = static_cast<unsigned char *>(p);
    return EPIC_OK;
}

}  // namespace

extern "C" int epic_geodesic_labels_noalloc(const float *cost_map, const float *matches,
                                            int H, int W, int N, int *labels_out,
                                            float *dist_out, void *stream_) {
    if (!cost_map || !matches || (!labels_out && !dist_out)) return EPIC_ERR_INVALID;
    if (H < 1 || W < 1 || N < 1) return EPIC_ERR_INVALID;
    if (((uintptr_t)matches % 16) != 0) return EPIC_ERR_INVALID;
    const long long P = (long long)H * W;
    const long long tiles_x = (W + NA_TILE_W - 1) / NA_TILE_W;
    const long long tiles_y = (H + NA_TILE_H - 1) / NA_TILE_H;
    if (P > NA_MAX_PIXELS || N > NA_MAX_MATCHES || tiles_x * tiles_y > NA_MAX_TILES)
        return EPIC_ERR_CAPACITY;
    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    int dev = 0, num_sms = 0, smem_optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
        return EPIC_ERR_CUDA;

    epic::PairDev Pd{};
    Pd.C = cost_map;
    Pd.matches = reinterpret_cast<const float4 *>(matches);
    Pd.flow = nullptr;
    Pd.H = H;
    Pd.W = W;
    Pd.N = N;
    Pd.K = 1;
    Pd.a = 1.f;
    Pd.tile_w = NA_TILE_W;
    Pd.tile_h = NA_TILE_H;
    Pd.apron = NA_APRON;
    Pd.tiles_x = (int)tiles_x;
    Pd.tiles_y = (int)tiles_y;
    Pd.hash_cap = 0;
    Pd.keys = reinterpret_cast<pkey_t *>(base + OFF_KEYS);
    Pd.tile_start = reinterpret_cast<int *>(base + OFF_TSTART);
    Pd.tile_fill = reinterpret_cast<int *>(base + OFF_TFILL);
    Pd.tile_seeds = reinterpret_cast<int *>(base + OFF_TSEEDS);
    Pd.tile_stamp = reinterpret_cast<int *>(base + OFF_TSTAMP);
    Pd.deg = reinterpret_cast<int *>(base + OFF_DEG);
    Pd.wmin = reinterpret_cast<unsigned *>(base + OFF_WMIN);
    Pd.info = reinterpret_cast<int *>(base + OFF_INFO);
    epic::RunState *state = reinterpret_cast<epic::RunState *>(base + OFF_STATE);
    // prefix arrays of a one-pair batch: {0, count}
    const int T = (int)(tiles_x * tiles_y);
    const int prefix[10] = {0, T, 0, N, 0, 0, 0, 0, 0, 0};
    if (cudaMemcpyAsync(base + OFF_PAIR, &Pd, sizeof(Pd), cudaMemcpyHostToDevice, stream) ||
        cudaMemcpyAsync(base + OFF_PREFIX, prefix, sizeof(prefix), cudaMemcpyHostToDevice,
                        stream) ||
        // the run state (status, pass counters, barrier) starts at zero
        cudaMemsetAsync(state, 0, sizeof(epic::RunState), stream))
        return EPIC_ERR_CUDA;
    // (copies from pageable host memory have consumed their source by the
    // time cudaMemcpyAsync returns)
    const int *pre = reinterpret_cast<const int *>(base + OFF_PREFIX);
    epic::BatchArgs a{};
    a.pairs = reinterpret_cast<const epic::PairDev *>(base + OFF_PAIR);
    a.npairs = 1;
    a.tile_base = pre + 0;
    a.match_base = pre + 2;
    a.chunk_base = pre + 4;
    a.hash_base = pre + 6;
    a.clear_base = pre + 8;
    a.total_tiles = T;
    a.total_matches = N;
    a.total_chunks = 0;
    a.total_hash = 0;
    a.total_clear = 0;
    a.max_degree = 1;
    a.max_passes = 4096;
    a.weight_squared = 1;
    a.fallback_eps = 1e-10f;
    a.state = state;
    const epic::BatchArgs *dev_a = reinterpret_cast<const epic::BatchArgs *>(base + OFF_ARGS);
    if (cudaMemcpyAsync(base + OFF_ARGS, &a, sizeof(a), cudaMemcpyHostToDevice, stream))
        return EPIC_ERR_CUDA;
    epic::LaunchCfg lc{num_sms, smem_optin, stream};
    if (epic::launch_prepare(a, dev_a, lc) != cudaSuccess ||
        epic::launch_dt(a, dev_a, lc, NA_TILE_W, NA_TILE_H, NA_APRON, false, nullptr) !=
            cudaSuccess ||
        epic::launch_split_keys(&Pd, reinterpret_cast<const epic::PairDev *>(base + OFF_PAIR),
                                labels_out, dist_out, stream) != cudaSuccess)
        return EPIC_ERR_CUDA;
    int status = 0;
    if (cudaMemcpyAsync(&status, &state->status, sizeof(int), cudaMemcpyDeviceToHost, stream) ||
        cudaStreamSynchronize(stream))
        return EPIC_ERR_CUDA;
    return status;
}
