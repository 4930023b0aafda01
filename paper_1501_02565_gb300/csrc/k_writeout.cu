// Stage (d): dense write-out (Algorithm 1 steps 7-8, LA form).
//
// Every pixel p takes the model of its cell's match m = L(p):
//     flow(p) = F(p) - p = c_m + B_m (p - p_m).
// The kernel is a single pass over the packed keys (8 B in, of which the
// label is the 4 B the method needs) and the flow (8 B out) of every pixel of
// the batch, so it is bound by HBM bandwidth:
//   * a work item is WRITEOUT_CHUNK pixels of one pair; each CTA takes a
//     contiguous run of items, two at a time (one per half of the CTA), so
//     the pair of an item is found once per run and followed forward;
//   * a warp handles 256 consecutive pixels as four rounds of 64: in each
//     round lane l takes pixels 2l and 2l + 1, so every key load and every
//     flow store (16 bytes a lane) of the warp is one contiguous run of 512
//     bytes; all four key loads are issued before the first model gather;
//   * the model table (32 bytes per match, a few MB for a batch) is read
//     through the read-only path, where it stays cache resident; flows are
//     written with streaming stores.
// The grid is one resident wave.
#include "epic_internal.cuh"

namespace epic {

namespace {

constexpr int WO_THREADS = 256;
constexpr int WO_GROUP = 128;   // threads per work item (four warps of 256 pixels)
static_assert(WRITEOUT_CHUNK == (WO_GROUP / 32) * 256, "a work item is four warps' pixels");

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
        // this warp's 256 pixels of the item
        const long long pw = (long long)(c - __ldg(chunk_base + pi)) * WRITEOUT_CHUNK +
                             (long long)(gt >> 5) * 256;
        if (pw >= npix) continue;
        const int lane = gt & 31;
        const pkey_t *keys = P.keys;
        const float4 *models = P.models;
        float *flow = P.flow;
        if (P.flow_vec_ok && pw + 256 <= npix) {
            ulonglong2 k[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                k[i] = __ldcs(reinterpret_cast<const ulonglong2 *>(keys + pw + 64 * i + 2 * lane));
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const long long q = pw + 64 * i + 2 * lane;
                int y = (int)(q / W), x = (int)(q - (long long)y * W);
                const float2 v0 = apply(models, key_label(k[i].x), N, x, y);
                if (++x == W) { x = 0; ++y; }
                const float2 v1 = apply(models, key_label(k[i].y), N, x, y);
                __stcs(reinterpret_cast<float4 *>(flow + 2 * q), make_float4(v0.x, v0.y, v1.x, v1.y));
            }
        } else {
            for (long long q = pw + lane; q < pw + 256 && q < npix; q += 32) {
                const int y = (int)(q / W), x = (int)(q - (long long)y * W);
                const float2 v = apply(models, key_label(__ldg(keys + q)), N, x, y);
                flow[2 * q] = v.x;
                flow[2 * q + 1] = v.y;
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
