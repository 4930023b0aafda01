// Per-run preparation: seed binning and scratch clearing.
//
// * Seeds of the assignment map (Sec. 3.4: every match p_m is at distance 0
//   from itself) are grouped by relaxation tile, so a tile's first solve can
//   place the seeds that fall inside its region without scanning all N
//   matches.  A match's source pixel is (floor(x+0.5), floor(y+0.5)); one
//   outside the image is an invalid input and sets EPIC_ERR_INVALID.
// * The match-graph edge table, the node degrees and lightest edges are
//   reset so that the graph stage can insert with atomics.
// * The run's grid-barrier and pass counters are reset.
#include "epic_internal.cuh"

namespace epic {

namespace {

// Exclusive scan of v[0..n) in place, by one CTA; v[n] receives the total.
__device__ void block_exclusive_scan(int *v, int n) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = blockDim.x >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        int i = base + tid;
        int x = (i < n) ? v[i] : 0;
        int s = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane == 31) warp_sums[wid] = s;
        __syncthreads();
        if (wid == 0) {
            int ws = (lane < nw) ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += t;
            }
            warp_sums[lane] = ws;  // inclusive prefix of warp totals
        }
        __syncthreads();
        int excl = carry + s - x + (wid > 0 ? warp_sums[wid - 1] : 0);
        if (i < n) v[i] = excl;
        __syncthreads();
        if (tid == blockDim.x - 1) carry = excl + x;
        __syncthreads();
    }
    if (tid == 0) v[n] = carry;
    __syncthreads();
}

__device__ __forceinline__ bool seed_pixel(float4 mt, int H, int W, int *px,
                                           int *py) {
    float fx = floorf(mt.x + 0.5f), fy = floorf(mt.y + 0.5f);
    if (!(fx >= 0.f && fx < (float)W && fy >= 0.f && fy < (float)H))
        return false;
    *px = (int)fx;
    *py = (int)fy;
    return true;
}

__global__ void __launch_bounds__(1024) prepare_kernel(const BatchArgs *__restrict__ ap) {
    const BatchArgs a = *ap;
    RunState *st = a.state;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // Nothing else touches these until the relaxation kernel starts,
        // which is stream-ordered after this one.
        st->passes = 0;
        st->changed[0] = st->changed[1] = st->changed[2] = 0;
        st->work[0] = st->work[1] = st->work[2] = st->work[3] = 0;
        st->knn_next = 0;
        st->knn_overflow = 0;
        st->knn_retry = 0;
        st->edge_next = 0;
        st->wl_count[0] = st->wl_count[1] = st->wl_count[2] = 0;
        st->barrier.count = 0;
        st->compact_done = 0;
    }
    // seed binning: one CTA per pair at a time
    for (int p = blockIdx.x; p < a.npairs; p += gridDim.x) {
        const PairDev &P = a.pairs[p];
        const int T = P.tiles_x * P.tiles_y;
        for (int t = threadIdx.x; t < T; t += blockDim.x) P.tile_start[t] = 0;
        for (int m = threadIdx.x; m < P.N; m += blockDim.x) {
            P.deg[m] = 0;
            P.wmin[m] = 0x7F800000u;  // +inf
        }
        if (threadIdx.x < 4) P.info[threadIdx.x] = 0;
        __syncthreads();
        for (int m = threadIdx.x; m < P.N; m += blockDim.x) {
            int x, y;
            if (!seed_pixel(P.matches[m], P.H, P.W, &x, &y)) {
                set_status(st, EPIC_ERR_INVALID);
                continue;
            }
            atomicAdd(&P.tile_start[(y / P.tile_h) * P.tiles_x + x / P.tile_w], 1);
        }
        __syncthreads();
        block_exclusive_scan(P.tile_start, T);
        for (int t = threadIdx.x; t < T; t += blockDim.x)
            P.tile_fill[t] = P.tile_start[t];
        __syncthreads();
        for (int m = threadIdx.x; m < P.N; m += blockDim.x) {
            int x, y;
            if (!seed_pixel(P.matches[m], P.H, P.W, &x, &y)) continue;
            int t = (y / P.tile_h) * P.tiles_x + x / P.tile_w;
            P.tile_seeds[atomicAdd(&P.tile_fill[t], 1)] = m;
        }
        __syncthreads();
    }
    // clearing: edge table slots, CLEAR_CHUNK items each (the CSR adjacency
    // is written in full by the scatter and needs no clearing)
    for (int c = blockIdx.x; c < a.total_clear; c += gridDim.x) {
        int p = find_pair(a.clear_base, a.npairs, c);
        const PairDev &P = a.pairs[p];
        long long i0 = (long long)(c - a.clear_base[p]) * CLEAR_CHUNK;
        long long n_hash = P.hash_cap;
        for (long long i = i0 + threadIdx.x; i < i0 + CLEAR_CHUNK && i < n_hash; i += blockDim.x) {
            P.hkeys[i] = EMPTY64;
            P.hw[i] = 0xFFFFFFFFu;
        }
    }
}

}  // namespace

cudaError_t launch_prepare(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc) {
    (void)a;
    int grid = lc.num_sms * 2;
    prepare_kernel<<<grid, 1024, 0, lc.stream>>>(dev);
    return cudaGetLastError();
}

}  // namespace epic
