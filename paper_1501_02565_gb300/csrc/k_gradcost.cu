// Cost map from the image gradient (Table 2, the "||grad_2 I||_2" contour
// row): C(p) = floor + sqrt(sum_c gx_c^2 + gy_c^2) with central differences
// gx = (I(x+1) - I(x-1)) / 2 on the edge-replicated image.
//
// A stack of frames [F][H][W][channels] float32 is processed in one launch,
// one thread per pixel; each frame's borders are its own.  The kernel is a
// 5-point stencil: every input value is used by five threads, which the
// warp's contiguous loads and L1/L2 serve, so DRAM sees each input byte and
// each output byte about once (channels * 4 + 4 bytes per pixel).
#include "epic_internal.cuh"

namespace epic {

namespace {

template <int CH>
__global__ void __launch_bounds__(256) gradcost_kernel(const float *__restrict__ img, int F, int H,
                                                       int W, float floor_, float *__restrict__ C) {
    const long long HW = (long long)H * W, n = HW * F;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long f = i / HW, r = i - f * HW;
        const int y = (int)(r / W), x = (int)(r - (long long)y * W);
        const float *fr = img + f * HW * CH;
        const long long xl = (long long)y * W + (x > 0 ? x - 1 : x);
        const long long xr = (long long)y * W + (x < W - 1 ? x + 1 : x);
        const long long yu = (long long)(y > 0 ? y - 1 : y) * W + x;
        const long long yd = (long long)(y < H - 1 ? y + 1 : y) * W + x;
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const float gx = __fmul_rn(__fsub_rn(__ldg(fr + xr * CH + c), __ldg(fr + xl * CH + c)), 0.5f);
            const float gy = __fmul_rn(__fsub_rn(__ldg(fr + yd * CH + c), __ldg(fr + yu * CH + c)), 0.5f);
            s = __fmaf_rn(gx, gx, s);
            s = __fmaf_rn(gy, gy, s);
        }
        __stcs(C + i, __fadd_rn(floor_, __fsqrt_rn(s)));
    }
}

}  // namespace

cudaError_t launch_gradcost(const float *img, int F, int H, int W, int channels, float floor_,
                            float *C, int num_sms, cudaStream_t stream) {
    const long long n = (long long)F * H * W;
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)num_sms * 8;   // 8 resident CTAs of 256 per SM
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    switch (channels) {
    case 1: gradcost_kernel<1><<<(unsigned)blocks, 256, 0, stream>>>(img, F, H, W, floor_, C); break;
    case 3: gradcost_kernel<3><<<(unsigned)blocks, 256, 0, stream>>>(img, F, H, W, floor_, C); break;
    case 4: gradcost_kernel<4><<<(unsigned)blocks, 256, 0, stream>>>(img, F, H, W, floor_, C); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace epic
