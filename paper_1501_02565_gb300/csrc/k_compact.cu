// Consistency pruning between two passes (Sec. 4.1 "Pruning of matches": the
// interpolation is run once with the Nadaraya-Watson estimator and the
// matches farther than a threshold from that estimate are removed).
//
// The first pass leaves keep[m] per match.  compact_kernel (one CTA per
// pair) writes the kept matches, in their original order, to the pair's
// scratch copy and rewrites the pair's device descriptor: matches -> the
// copy, N -> the kept count, K -> min(K of the second pass, kept count).  If
// nothing is kept the pair keeps all its matches.  A last CTA rebuilds the
// batch's match prefix sums and switches the estimator for the second pass,
// so the second pass reads everything from device memory and needs no host
// round trip.
#include "epic_internal.cuh"

namespace epic {

namespace {

__device__ int block_scan_exclusive(int x, int *total) {
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int s = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
    }
    if (lane == 31) warp_sums[wid] = s;
    __syncthreads();
    if (wid == 0) {
        int ws = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += t;
        }
        warp_sums[lane] = ws;
    }
    __syncthreads();
    const int excl = s - x + (wid > 0 ? warp_sums[wid - 1] : 0);
    *total = warp_sums[nw - 1];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(1024) compact_kernel(BatchArgs *ap, unsigned *done) {
    const BatchArgs a = *ap;
    if (get_status(a.state) != 0) return;
    PairDev *pairs = const_cast<PairDev *>(a.pairs);
    __shared__ int s_kept;
    for (int p = blockIdx.x; p < a.npairs; p += gridDim.x) {
        PairDev &P = pairs[p];
        const int n = P.N;
        // count the kept matches
        int kept = 0;
        for (int i0 = 0; i0 < n; i0 += blockDim.x) {
            const int i = i0 + threadIdx.x;
            kept += __syncthreads_count(i < n && P.keep[i] != 0);
        }
        // write them in their original order (all of them if none is kept)
        const bool all = kept == 0;
        int base = 0;
        for (int i0 = 0; i0 < n; i0 += blockDim.x) {
            const int i = i0 + threadIdx.x;
            const int k = i < n && (all || P.keep[i] != 0) ? 1 : 0;
            int tot;
            const int pos = base + block_scan_exclusive(k, &tot);
            if (k) {
                P.pruned[pos] = P.matches[i];
                P.kept_index[pos] = i;
            }
            base += tot;
        }
        if (threadIdx.x == 0) s_kept = base;
        __syncthreads();
        if (threadIdx.x == 0) {
            const int nk = s_kept;
            P.matches = P.pruned;
            P.N = nk;
            P.K = min(P.K2, nk);
        }
        __syncthreads();
    }
    // the last CTA to finish rebuilds the match prefix sums
    __shared__ bool s_last;
    __threadfence();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        int *mb = const_cast<int *>(a.match_base);
        int acc = 0;
        for (int p = 0; p < a.npairs; ++p) {
            mb[p] = acc;
            acc += *(volatile int *)&pairs[p].N;
        }
        mb[a.npairs] = acc;
        ap->total_matches = acc;
        ap->estimator = a.final_estimator;
        ap->write_keep = 0;
        *done = 0;  // ready for the next run
    }
}

}  // namespace

cudaError_t launch_compact(const BatchArgs &a, BatchArgs *dev, const LaunchCfg &lc) {
    int grid = a.npairs < lc.num_sms ? a.npairs : lc.num_sms;
    if (grid < 1) grid = 1;
    compact_kernel<<<grid, 1024, 0, lc.stream>>>(dev, &a.state->compact_done);
    return cudaGetLastError();
}

}  // namespace epic
