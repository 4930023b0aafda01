// Cost map from the image gradient (Table 2, the "||grad_2 I||_2" contour
// row): C(p) = floor + sqrt(sum_c gx_c^2 + gy_c^2) with central differences
// gx = (I(x+1) - I(x-1)) / 2 on the edge-replicated image.
//
// A stack of frames [F][H][W][channels] float32 is processed in one launch;
// each frame's borders are its own.  The algorithmic traffic is one read of
// the image and one write of the cost (channels * 4 + 4 bytes per pixel).
#include "epic_internal.cuh"

namespace epic {

namespace {

constexpr int GC_THREADS = 256;   // columns per CTA
constexpr int GC_ROWS = 8;        // rows per CTA (a tile of one frame)

// A CTA computes a tile of GC_ROWS x GC_THREADS pixels of one frame.  It
// copies the tile plus a one-pixel halo into shared memory with contiguous
// 4-byte loads (consecutive threads read consecutive floats of a row, so
// every load instruction covers whole sectors), all issued before any is
// stored so that each thread has ~(GC_ROWS + 2) * 3 loads in flight; the
// halo is clamped to the frame, which is the edge replication.  Then each
// thread computes its column's GC_ROWS pixels from shared memory.  DRAM
// reads each input byte about once; L2 sees (GC_ROWS + 2) / GC_ROWS of it.
template <int CH>
__device__ __forceinline__ void gradcost_tile(const float *__restrict__ img, int H, int W,
                                              int tiles_per_frame, int tile, float floor_,
                                              float *__restrict__ C, float *sm) {
    constexpr int SW = (GC_THREADS + 2) * CH;   // floats per staged row
    constexpr int PER = (SW + GC_THREADS - 1) / GC_THREADS;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * GC_THREADS;
    const int f = tile / tiles_per_frame;
    const int y0 = (tile - f * tiles_per_frame) * GC_ROWS;
    const float *fr = img + (size_t)f * H * W * CH;
    float v[GC_ROWS + 2][PER];
#pragma unroll
    for (int r = 0; r < GC_ROWS + 2; ++r) {
        const int y = min(max(y0 - 1 + r, 0), H - 1);
        const float *row = fr + (size_t)y * W * CH;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = t + k * GC_THREADS;
            const int col = min(max(x0 - 1 + i / CH, 0), W - 1);
            v[r][k] = i < SW ? __ldg(row + (size_t)col * CH + i % CH) : 0.f;
        }
    }
    __syncthreads();   // the previous tile's reads of sm are done
#pragma unroll
    for (int r = 0; r < GC_ROWS + 2; ++r)
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = t + k * GC_THREADS;
            if (i < SW) sm[r * SW + i] = v[r][k];
        }
    __syncthreads();
    const int x = x0 + t;
    if (x >= W) return;
    float *out = C + (size_t)f * H * W;
    for (int r = 0; r < GC_ROWS && y0 + r < H; ++r) {
        const float *up = sm + r * SW, *mid = up + SW, *dn = mid + SW;
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const float gx = __fmul_rn(__fsub_rn(mid[(t + 2) * CH + c], mid[t * CH + c]), 0.5f);
            const float gy = __fmul_rn(__fsub_rn(dn[(t + 1) * CH + c], up[(t + 1) * CH + c]), 0.5f);
            s = __fmaf_rn(gx, gx, s);
            s = __fmaf_rn(gy, gy, s);
        }
        __stcs(out + (size_t)(y0 + r) * W + x, __fadd_rn(floor_, __fsqrt_rn(s)));
    }
}

template <int CH>
__global__ void __launch_bounds__(GC_THREADS) gradcost_kernel(const float *__restrict__ img, int H,
                                                              int W, int tiles_per_frame,
                                                              int tiles, float floor_,
                                                              float *__restrict__ C) {
    __shared__ float sm[(GC_ROWS + 2) * (GC_THREADS + 2) * CH];
    for (int s = blockIdx.y; s < tiles; s += gridDim.y)
        gradcost_tile<CH>(img, H, W, tiles_per_frame, s, floor_, C, sm);
}

}  // namespace

cudaError_t launch_gradcost(const float *img, int F, int H, int W, int channels, float floor_,
                            float *C, int num_sms, cudaStream_t stream) {
    (void)num_sms;
    const int spf = (H + GC_ROWS - 1) / GC_ROWS;
    const long long total = (long long)F * spf;
    if (total > 2147483647LL) return cudaErrorInvalidValue;
    const int n = (int)total;
    const dim3 grid((W + GC_THREADS - 1) / GC_THREADS, (unsigned)(n < 65535 ? n : 65535));
    switch (channels) {
    case 1: gradcost_kernel<1><<<grid, GC_THREADS, 0, stream>>>(img, H, W, spf, n, floor_, C); break;
    case 3: gradcost_kernel<3><<<grid, GC_THREADS, 0, stream>>>(img, H, W, spf, n, floor_, C); break;
    case 4: gradcost_kernel<4><<<grid, GC_THREADS, 0, stream>>>(img, H, W, spf, n, floor_, C); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace epic
