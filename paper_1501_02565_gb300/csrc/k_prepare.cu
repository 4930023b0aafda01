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
// * For the warp-tile relaxation, each pair's largest cost and the reach of
//   its seeds over the tile grid (a Chebyshev distance transform of the
//   seeded tiles) are recorded; they fix the pair's distance unit (see
//   unit_shift in epic_internal.cuh).
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

// Chebyshev distance, in tile steps, from every tile to the nearest tile
// holding a seed (the scatter cursors, no longer needed, are the scratch),
// and its largest value in P.seed_reach.  One CTA per pair.
__device__ void seed_reach(const PairDev &P, int T) {
    __shared__ int s_changed;
    int *d = P.tile_fill;
    for (int t = threadIdx.x; t < T; t += blockDim.x)
        d[t] = P.tile_start[t + 1] > P.tile_start[t] ? 0 : 0x3fffffff;
    __syncthreads();
    // at most max(tiles_x, tiles_y) rounds: every round extends the distances by a tile
    for (int round = 0; round <= max(P.tiles_x, P.tiles_y); ++round) {
        if (threadIdx.x == 0) s_changed = 0;
        __syncthreads();
        for (int t = threadIdx.x; t < T; t += blockDim.x) {
            const int tx = t % P.tiles_x, ty = t / P.tiles_x;
            int best = d[t];
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int x = tx + dx, y = ty + dy;
                    if (x >= 0 && x < P.tiles_x && y >= 0 && y < P.tiles_y)
                        best = min(best, *(volatile int *)&d[y * P.tiles_x + x] + 1);
                }
            if (best < d[t]) {
                d[t] = best;
                s_changed = 1;
            }
        }
        __syncthreads();
        if (!s_changed) break;
        __syncthreads();
    }
    int far = 0;
    for (int t = threadIdx.x; t < T; t += blockDim.x) far = max(far, d[t]);
    far = __reduce_max_sync(0xffffffffu, far);
    __shared__ int s_far;
    if (threadIdx.x == 0) s_far = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&s_far, far);
    __syncthreads();
    if (threadIdx.x == 0) const_cast<PairDev &>(P).seed_reach = s_far;
    __syncthreads();
}

// Largest cost of every warp-tile pair (float bits; costs are >= 0, so the
// bits order like the values, and a NaN or negative cost shows as a value
// above +inf).  Work items are the write-out chunks (1024 pixels); each CTA
// takes a contiguous run, its four groups of 256 threads an item at a time
// (four pixels a thread), and a warp's running maximum goes out with one
// atomic whenever its pair changes.
__device__ void cost_max(const BatchArgs &a) {
    // the CTAs that binned a pair's seeds take no part when enough others
    // are left (they would finish last)
    const int first = a.npairs < (int)gridDim.x / 2 ? a.npairs : 0;
    if ((int)blockIdx.x < first) return;
    const int nb = (int)gridDim.x - first, b = (int)blockIdx.x - first;
    const int per = (a.total_chunks + nb - 1) / nb;
    const int c0 = b * per, c1 = min(a.total_chunks, c0 + per);
    const int grp = threadIdx.x >> 8, gt = threadIdx.x & 255;   // warp-uniform group
    int pi = -1;
    unsigned mx = 0;
    auto flush = [&]() {
        const unsigned wm = __reduce_max_sync(0xffffffffu, mx);
        if (pi >= 0 && (threadIdx.x & 31) == 0)
            atomicMax(const_cast<unsigned *>(&a.pairs[pi].cmax_bits), wm);
        mx = 0;
    };
    for (int c = c0 + grp; c < c1; c += 4) {
        const int p = find_pair(a.chunk_base, a.npairs, c);
        if (p != pi) {
            flush();
            pi = p;
        }
        const PairDev &P = a.pairs[p];
        if (P.sweep != SWEEP_WARP) continue;
        const long long npx = (long long)P.H * P.W;
        const long long i = (long long)(c - a.chunk_base[p]) * WRITEOUT_CHUNK + 4 * gt;
        if (i + 3 < npx && ((uintptr_t)P.C & 15) == 0) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(P.C + i));
            mx = max(max(mx, __float_as_uint(v.x)), max(__float_as_uint(v.y), max(
                         __float_as_uint(v.z), __float_as_uint(v.w))));
        } else {
            for (int j = 0; j < 4 && i + j < npx; ++j)
                mx = max(mx, __float_as_uint(__ldg(P.C + i + j)));
        }
    }
    flush();
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
        st->q_head = st->q_tail = st->q_items = 0;
        st->q_busy = a.total_tiles;   // the initial sweep's items
    }
    // the warp-tile relaxation's work queue: empty slots; every tile counts
    // as queued until the sweep of phase 2 takes it.  Runs of the apron-tile
    // relaxation (the exact variant's, the no-allocation entry point's) have
    // no queue.
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; a.relax_queue && i < a.total_tiles;
         i += gridDim.x * blockDim.x) {
        a.relax_queue[i] = -1;
        a.relax_queued[i] = 1;
    }
    // seed binning: one CTA per pair at a time
    for (int p = blockIdx.x; p < a.npairs; p += gridDim.x) {
        const PairDev &P = a.pairs[p];
        const int T = P.tiles_x * P.tiles_y;
        for (int t = threadIdx.x; t < T; t += blockDim.x) {
            P.tile_start[t] = 0;
            if (P.sweep == SWEEP_WARP) P.tile_stamp[t] = STAMP_PENDING;
        }
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
        if (P.sweep == SWEEP_WARP) seed_reach(P, T);
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
    cost_max(a);
}

}  // namespace

cudaError_t launch_prepare(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc) {
    (void)a;
    int grid = lc.num_sms * 2;
    prepare_kernel<<<grid, 1024, 0, lc.stream>>>(dev);
    return cudaGetLastError();
}

}  // namespace epic
