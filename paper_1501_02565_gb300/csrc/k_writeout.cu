// Stage (d): dense write-out (Algorithm 1 steps 7-8, LA form).
//
// Every pixel p takes the model of its cell's match m = L(p):
//     flow(p) = F(p) - p = c_m + B_m (p - p_m).
// The kernel is a single pass over the labels (4 B in, the plane the edge
// stage writes beside the packed keys) and the flow (8 B out) of every pixel
// of the batch, so it is bound by HBM bandwidth:
//   * a work item is WRITEOUT_CHUNK pixels of one pair; each CTA takes a
//     contiguous run of items, two at a time (one per half of the CTA), so
//     the pair of an item is found once per run and followed forward;
//   * a thread handles eight consecutive pixels: its two 16-byte label loads
//     are issued before the first model gather;
//   * the model table (32 bytes per match, a few MB for a batch) is read
//     through the read-only path, where it stays cache resident; flows are
//     written with streaming 16-byte stores.
// The grid is one resident wave.
#include "epic_internal.cuh"

namespace epic {

namespace {

constexpr int WO_THREADS = 256;
constexpr int WO_GROUP = 128;   // threads per work item
constexpr int WO_PER_THREAD = WRITEOUT_CHUNK / WO_GROUP;
static_assert(WO_PER_THREAD == 8, "eight pixels per thread");

__device__ __forceinline__ float2 apply(const float4 *models, unsigned m, int n, int x,
                                        int y) {
    if (m >= (unsigned)n) return make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
    const float4 r0 = __ldg(models + 2 * (size_t)m);
    const float4 r1 = __ldg(models + 2 * (size_t)m + 1);
    const float dx = (float)x - r1.z, dy = (float)y - r1.w;
    return make_float2(r0.x + r0.z * dx + r0.w * dy, r0.y + r1.x * dx + r1.y * dy);
}

__global__ void __launch_bounds__(WO_THREADS) writeout_kernel(const BatchArgs *__restrict__ ap) {
    RunState *st = ap->state;
    if (get_status(st) != 0) return;
    const PairDev *pairs = ap->pairs;
    const int *chunk_base = ap->chunk_base;
    const int npairs = ap->npairs, total = ap->total_chunks;
    const int grp = threadIdx.x / WO_GROUP, gt = threadIdx.x % WO_GROUP;
    // contiguous runs of items per CTA; the two halves take alternate items
    const int per = ((total + gridDim.x - 1) / gridDim.x + 1) & ~1;
    const int c0 = blockIdx.x * per, c1 = min(total, c0 + per);
    if (c0 + grp >= c1) return;
    int pi = find_pair(chunk_base, npairs, c0 + grp);
    int next_base = __ldg(chunk_base + pi + 1);
    for (int c = c0 + grp; c < c1; c += 2) {
        while (c >= next_base) {
            ++pi;
            next_base = __ldg(chunk_base + pi + 1);
        }
        const PairDev &P = pairs[pi];
        const int W = P.W, N = P.N;
        const long long npix = (long long)P.H * W;
        const long long p0 = (long long)(c - __ldg(chunk_base + pi)) * WRITEOUT_CHUNK +
                             (long long)gt * WO_PER_THREAD;
        if (p0 >= npix) continue;
        const unsigned *labels = P.labels;
        const float4 *models = P.models;
        float *flow = P.flow;
        int y = (int)(p0 / W), x = (int)(p0 - (long long)y * W);
        if (P.flow_vec_ok && p0 + WO_PER_THREAD <= npix) {
            const uint4 l0 = __ldcs(reinterpret_cast<const uint4 *>(labels + p0));
            const uint4 l1 = __ldcs(reinterpret_cast<const uint4 *>(labels + p0) + 1);
            const unsigned ls[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
            float4 o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 v0 = apply(models, ls[2 * i], N, x, y);
                if (++x == W) { x = 0; ++y; }
                const float2 v1 = apply(models, ls[2 * i + 1], N, x, y);
                if (++x == W) { x = 0; ++y; }
                o[i] = make_float4(v0.x, v0.y, v1.x, v1.y);
            }
            float4 *out = reinterpret_cast<float4 *>(flow + 2 * p0);
#pragma unroll
            for (int i = 0; i < 4; ++i) __stcs(out + i, o[i]);
        } else {
            for (int i = 0; i < WO_PER_THREAD && p0 + i < npix; ++i) {
                const float2 v = apply(models, __ldg(labels + p0 + i), N, x, y);
                flow[2 * (p0 + i)] = v.x;
                flow[2 * (p0 + i) + 1] = v.y;
                if (++x == W) { x = 0; ++y; }
            }
        }
    }
}

}  // namespace

cudaError_t launch_writeout(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc) {
    (void)a;
    int per_sm = 0;
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, writeout_kernel, WO_THREADS, 0);
    if (e != cudaSuccess) return e;
    writeout_kernel<<<lc.num_sms * (per_sm > 0 ? per_sm : 1), WO_THREADS, 0, lc.stream>>>(dev);
    return cudaGetLastError();
}

}  // namespace epic
