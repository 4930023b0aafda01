// Stage (d): dense write-out (Algorithm 1 steps 7-8, LA form).
//
// Every pixel p takes the model of its cell's match m = L(p):
//     flow(p) = F(p) - p = c_m + B_m (p - p_m).
// A work item is WRITEOUT_CHUNK consecutive pixels of one pair; a thread
// handles four consecutive pixels with two 16-byte key loads and two 16-byte
// streaming flow stores.  The model table (32 bytes per match) is small and
// read through the read-only path, where it stays cache resident.
#include "epic_internal.cuh"

namespace epic {

namespace {

__device__ __forceinline__ float2 apply(const float4 *models, unsigned m, int n, int x,
                                        int y) {
    if (m >= (unsigned)n) return make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
    const float4 r0 = __ldg(models + 2 * (size_t)m);
    const float4 r1 = __ldg(models + 2 * (size_t)m + 1);
    const float dx = (float)x - r1.z, dy = (float)y - r1.w;
    return make_float2(r0.x + r0.z * dx + r0.w * dy, r0.y + r1.x * dx + r1.y * dy);
}

__device__ __forceinline__ void st_stream(float4 *p, float4 v) { __stcs(p, v); }

__global__ void __launch_bounds__(256) writeout_kernel(const BatchArgs *__restrict__ ap) {
    const BatchArgs a = *ap;
    RunState *st = a.state;
    if (get_status(st) != 0) return;
    constexpr int PER_THREAD = WRITEOUT_CHUNK / 256;
    static_assert(PER_THREAD == 4, "four pixels per thread");
    for (int c = blockIdx.x; c < a.total_chunks; c += gridDim.x) {
        const int pi = find_pair(a.chunk_base, a.npairs, c);
        const PairDev &P = a.pairs[pi];
        const long long npix = (long long)P.H * P.W;
        const long long p0 = (long long)(c - a.chunk_base[pi]) * WRITEOUT_CHUNK +
                             (long long)threadIdx.x * PER_THREAD;
        if (p0 >= npix) continue;
        int y = (int)(p0 / P.W), x = (int)(p0 - (long long)y * P.W);
        if (P.flow_vec_ok && p0 + 3 < npix) {
            const ulonglong2 k01 = __ldg(reinterpret_cast<const ulonglong2 *>(P.keys + p0));
            const ulonglong2 k23 = __ldg(reinterpret_cast<const ulonglong2 *>(P.keys + p0 + 2));
            const pkey_t ks[4] = {k01.x, k01.y, k23.x, k23.y};
            float f[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float2 v = apply(P.models, key_label(ks[i]), P.N, x, y);
                f[2 * i] = v.x;
                f[2 * i + 1] = v.y;
                if (++x == P.W) { x = 0; ++y; }
            }
            float4 *out = reinterpret_cast<float4 *>(P.flow + 2 * p0);
            st_stream(out, make_float4(f[0], f[1], f[2], f[3]));
            st_stream(out + 1, make_float4(f[4], f[5], f[6], f[7]));
        } else {
            for (int i = 0; i < 4 && p0 + i < npix; ++i) {
                const pkey_t k = __ldg(P.keys + p0 + i);
                float2 v = apply(P.models, key_label(k), P.N, x, y);
                P.flow[2 * (p0 + i)] = v.x;
                P.flow[2 * (p0 + i) + 1] = v.y;
                if (++x == P.W) { x = 0; ++y; }
            }
        }
    }
}

}  // namespace

cudaError_t launch_writeout(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc) {
    (void)a;
    writeout_kernel<<<lc.num_sms * 8, 256, 0, lc.stream>>>(dev);
    return cudaGetLastError();
}

}  // namespace epic
