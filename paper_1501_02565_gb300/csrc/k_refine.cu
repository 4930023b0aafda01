// Variational refinement (Sec. 4, "Variational Energy Minimization"): the
// interpolated flow is refined at full resolution by fixed-point iterations,
// each linearising the data term (colour and gradient constancy with
// normalisation) at the current flow and solving the linear system of the
// Euler-Lagrange equations for the update with red-black SOR.
//
// Per fixed-point iteration:
//   warp_kernel    I2w(p) = I2(p + w(p)), bilinear, coordinates clamped;
//   coeff_kernel   per pixel the 2x2 data matrix A, right-hand side b (with
//                  the robust weights taken at zero update) and the
//                  smoothness weight phi = alpha Psi'(|grad u|^2 + |grad v|^2);
//   sor_block_kernel  several half-sweeps (colours alternating) of
//                  point-coupled SOR on overlapped tiles in shared memory:
//                  the 2x2 system of (du, dv) at a pixel is solved exactly
//                  from the current neighbours and over-relaxed;
//   update_kernel  w += (du, dv).
// Derivatives are central differences on the edge-replicated image, nested
// the same way for second derivatives (the derivative image is itself
// edge-replicated).  All arithmetic is float32.
#include "epic_internal.cuh"

namespace epic {

namespace {

struct Img {
    const float *p;
    int H, W, C;
    __device__ __forceinline__ float at(int x, int y, int c) const {
        x = min(max(x, 0), W - 1);
        y = min(max(y, 0), H - 1);
        return __ldg(p + ((size_t)y * W + x) * C + c);
    }
    // D_x I at (x, y) for an in-image (x, y)
    __device__ __forceinline__ float gx(int x, int y, int c) const {
        return 0.5f * (at(x + 1, y, c) - at(x - 1, y, c));
    }
    __device__ __forceinline__ float gy(int x, int y, int c) const {
        return 0.5f * (at(x, y + 1, c) - at(x, y - 1, c));
    }
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

__global__ void warp_kernel(const float *__restrict__ I2, const float *__restrict__ flow, int H,
                            int W, int C, float *__restrict__ I2w) {
    const long long P = (long long)H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (long long)y * W);
        const float X = fminf(fmaxf((float)x + flow[2 * i], 0.f), (float)(W - 1));
        const float Y = fminf(fmaxf((float)y + flow[2 * i + 1], 0.f), (float)(H - 1));
        const int x0 = W > 1 ? min((int)floorf(X), W - 2) : 0;
        const int y0 = H > 1 ? min((int)floorf(Y), H - 2) : 0;
        const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
        const float ax = X - (float)x0, ay = Y - (float)y0;
        for (int c = 0; c < C; ++c) {
            const float a00 = __ldg(I2 + ((size_t)y0 * W + x0) * C + c);
            const float a01 = __ldg(I2 + ((size_t)y0 * W + x1) * C + c);
            const float a10 = __ldg(I2 + ((size_t)y1 * W + x0) * C + c);
            const float a11 = __ldg(I2 + ((size_t)y1 * W + x1) * C + c);
            I2w[i * C + c] = (1.f - ay) * ((1.f - ax) * a00 + ax * a01) +
                             ay * ((1.f - ax) * a10 + ax * a11);
        }
    }
}

__global__ void coeff_kernel(Img I1, Img I2w, const float *__restrict__ flow, RefineArgs r,
                             float *__restrict__ coef) {
    const int H = I1.H, W = I1.W, C = I1.C;
    const long long P = (long long)H * W;
    const float z2 = r.zeta * r.zeta, e2 = r.eps * r.eps;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (long long)y * W);
        const int xl = clampi(x - 1, 0, W - 1), xr = clampi(x + 1, 0, W - 1);
        const int yu = clampi(y - 1, 0, H - 1), yd = clampi(y + 1, 0, H - 1);
        float sc_t = 0.f, sg_t = 0.f;           // arguments of the two penalisers
        float c11 = 0.f, c12 = 0.f, c22 = 0.f, cb1 = 0.f, cb2 = 0.f;   // colour parts
        float g11 = 0.f, g12 = 0.f, g22 = 0.f, gb1 = 0.f, gb2 = 0.f;   // gradient parts
        float grad1 = 0.f;
        for (int c = 0; c < C; ++c) {
            const float g1x = I1.gx(x, y, c), g1y = I1.gy(x, y, c);
            const float g2x = I2w.gx(x, y, c), g2y = I2w.gy(x, y, c);
            grad1 += g1x * g1x + g1y * g1y;
            // colour constancy
            const float Ix = 0.5f * (g1x + g2x), Iy = 0.5f * (g1y + g2y);
            const float Iz = I2w.at(x, y, c) - I1.at(x, y, c);
            const float t0 = 1.f / (Ix * Ix + Iy * Iy + z2);
            sc_t += t0 * Iz * Iz;
            c11 += t0 * Ix * Ix; c12 += t0 * Ix * Iy; c22 += t0 * Iy * Iy;
            cb1 += t0 * Ix * Iz; cb2 += t0 * Iy * Iz;
            // gradient constancy: derivatives of the gradient images
            const float Ixx = 0.5f * (0.5f * (I1.gx(xr, y, c) - I1.gx(xl, y, c)) +
                                      0.5f * (I2w.gx(xr, y, c) - I2w.gx(xl, y, c)));
            const float Ixy = 0.5f * (0.5f * (I1.gx(x, yd, c) - I1.gx(x, yu, c)) +
                                      0.5f * (I2w.gx(x, yd, c) - I2w.gx(x, yu, c)));
            const float Iyx = 0.5f * (0.5f * (I1.gy(xr, y, c) - I1.gy(xl, y, c)) +
                                      0.5f * (I2w.gy(xr, y, c) - I2w.gy(xl, y, c)));
            const float Iyy = 0.5f * (0.5f * (I1.gy(x, yd, c) - I1.gy(x, yu, c)) +
                                      0.5f * (I2w.gy(x, yd, c) - I2w.gy(x, yu, c)));
            const float Ixz = g2x - g1x, Iyz = g2y - g1y;
            const float tx = 1.f / (Ixx * Ixx + Ixy * Ixy + z2);
            const float ty = 1.f / (Iyx * Iyx + Iyy * Iyy + z2);
            sg_t += tx * Ixz * Ixz + ty * Iyz * Iyz;
            g11 += tx * Ixx * Ixx + ty * Iyx * Iyx;
            g12 += tx * Ixx * Ixy + ty * Iyx * Iyy;
            g22 += tx * Ixy * Ixy + ty * Iyy * Iyy;
            gb1 += tx * Ixx * Ixz + ty * Iyx * Iyz;
            gb2 += tx * Ixy * Ixz + ty * Iyy * Iyz;
        }
        const float pc = 0.5f / sqrtf(sc_t + e2);
        const float pg = r.gamma * (0.5f / sqrtf(sg_t + e2));
        // smoothness: alpha(x) Psi'(|grad u|^2 + |grad v|^2), central differences
        const float *f = flow;
        const size_t il = (size_t)y * W + xl, ir = (size_t)y * W + xr;
        const size_t iu = (size_t)yu * W + x, id = (size_t)yd * W + x;
        const float ux = 0.5f * (f[2 * ir] - f[2 * il]), uy = 0.5f * (f[2 * id] - f[2 * iu]);
        const float vx = 0.5f * (f[2 * ir + 1] - f[2 * il + 1]);
        const float vy = 0.5f * (f[2 * id + 1] - f[2 * iu + 1]);
        const float alpha = r.alpha0 * expf(-r.kappa * sqrtf(grad1));
        const float phi = alpha * (0.5f / sqrtf(ux * ux + uy * uy + vx * vx + vy * vy + e2));
        float *o = coef + i * 8;
        o[0] = pc * c11 + pg * g11;
        o[1] = pc * c12 + pg * g12;
        o[2] = pc * c22 + pg * g22;
        o[3] = pc * cb1 + pg * gb1;
        o[4] = pc * cb2 + pg * gb2;
        o[5] = phi;
    }
}

// The point-coupled SOR update of one pixel from the neighbour sums
// S = sum s_pq, r1 = sum s_pq (u_q + du_q - u_p) (and r2 for v), each edge
// weight s_pq = (phi_p + phi_q) / 2; cp = (A11, A12, A22, b1, b2).  Returns
// false (no update) if the 2x2 system is not positive definite.
__device__ __forceinline__ bool sor_point(float S, float r1, float r2, float a11, float a12,
                                          float a22, float b1, float b2, float dup, float dvp,
                                          float omega, float &du, float &dv) {
    r1 -= b1;
    r2 -= b2;
    const float a = a11 + S, b = a12, dd = a22 + S;
    const float det = a * dd - b * b;
    if (!(det > 0.f)) return false;
    const float nu = (dd * r1 - b * r2) / det, nv = (a * r2 - b * r1) / det;
    du = (1.f - omega) * dup + omega * nu;
    dv = (1.f - omega) * dvp + omega * nv;
    return true;
}

// SOR_H half-sweeps per launch on overlapped tiles.  A CTA loads a region of
// (SOR_TX + 2 SOR_H) x (SOR_TY + 2 SOR_H) pixels (flow, update, coefficients)
// into shared memory and runs the half-sweeps there, red first.  Cells on
// the region's outer ring are never updated; a wrong value spreads inward by
// one pixel per half-sweep, so after SOR_H half-sweeps the core SOR_TX x
// SOR_TY pixels hold exactly what the half-sweeps over the whole image would
// give (each update is the same arithmetic on the same values).  The core is
// written to a second update buffer (the neighbours' halos still read the
// first), and the buffers swap between launches.
constexpr int SOR_TX = 32, SOR_TY = 32, SOR_H = 6;
constexpr int SOR_RW = SOR_TX + 2 * SOR_H, SOR_RH = SOR_TY + 2 * SOR_H, SOR_N = SOR_RW * SOR_RH;
constexpr size_t SOR_SMEM = 10 * SOR_N * sizeof(float);

__global__ void __launch_bounds__(256) sor_block_kernel(const float *__restrict__ flow,
                                                        const float *__restrict__ coef, int H,
                                                        int W, float omega, int nhalf,
                                                        const float *__restrict__ din,
                                                        float *__restrict__ dout) {
    extern __shared__ float sb[];
    float *su = sb, *sv = su + SOR_N, *sdu = sv + SOR_N, *sdv = sdu + SOR_N, *sph = sdv + SOR_N;
    float *sc = sph + SOR_N;   // 5 x SOR_N: A11, A12, A22, b1, b2
    const int rx0 = blockIdx.x * SOR_TX - SOR_H, ry0 = blockIdx.y * SOR_TY - SOR_H;
    for (int i = threadIdx.x; i < SOR_N; i += blockDim.x) {
        const int r = i / SOR_RW, c = i - r * SOR_RW;
        const int x = rx0 + c, y = ry0 + r;
        if (x < 0 || x >= W || y < 0 || y >= H) continue;
        const size_t p = (size_t)y * W + x;
        const float2 f = reinterpret_cast<const float2 *>(flow)[p];
        const float2 dd = reinterpret_cast<const float2 *>(din)[p];
        const float4 c0 = reinterpret_cast<const float4 *>(coef)[2 * p];
        const float4 c1 = reinterpret_cast<const float4 *>(coef)[2 * p + 1];
        su[i] = f.x;
        sv[i] = f.y;
        sdu[i] = dd.x;
        sdv[i] = dd.y;
        sph[i] = c1.y;
        sc[i] = c0.x;
        sc[SOR_N + i] = c0.y;
        sc[2 * SOR_N + i] = c0.z;
        sc[3 * SOR_N + i] = c0.w;
        sc[4 * SOR_N + i] = c1.x;
    }
    __syncthreads();
    static_assert(SOR_RW % 2 == 0, "a region row holds SOR_RW / 2 cells of each colour");
    constexpr int HALF_RW = SOR_RW / 2;
    for (int h = 0; h < nhalf; ++h) {
        const int colour = h & 1;
        // enumerate only this colour's cells: in row r they are the columns
        // c with (rx0 + c + ry0 + r) even (red) or odd (black)
        for (int k = threadIdx.x; k < SOR_RH * HALF_RW; k += blockDim.x) {
            const int r = k / HALF_RW;
            const int c = 2 * (k - r * HALF_RW) + ((colour + rx0 + ry0 + r) & 1);
            if (r == 0 || c == 0 || r == SOR_RH - 1 || c == SOR_RW - 1) continue;
            const int x = rx0 + c, y = ry0 + r;
            if (x < 0 || x >= W || y < 0 || y >= H) continue;
            const int i = r * SOR_RW + c;
            const float php = sph[i], up = su[i], vp = sv[i];
            float S = 0.f, r1 = 0.f, r2 = 0.f;
            auto nb = [&](int q) {   // right, left, down, up
                const float sw = 0.5f * (php + sph[q]);
                S += sw;
                r1 += sw * ((su[q] + sdu[q]) - up);
                r2 += sw * ((sv[q] + sdv[q]) - vp);
            };
            if (x + 1 < W) nb(i + 1);
            if (x > 0) nb(i - 1);
            if (y + 1 < H) nb(i + SOR_RW);
            if (y > 0) nb(i - SOR_RW);
            float du, dv;
            if (sor_point(S, r1, r2, sc[i], sc[SOR_N + i], sc[2 * SOR_N + i], sc[3 * SOR_N + i],
                          sc[4 * SOR_N + i], sdu[i], sdv[i], omega, du, dv)) {
                sdu[i] = du;
                sdv[i] = dv;
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < SOR_TX * SOR_TY; i += blockDim.x) {
        const int r = SOR_H + i / SOR_TX, c = SOR_H + i % SOR_TX;
        const int x = rx0 + c, y = ry0 + r;
        if (x >= W || y >= H) continue;
        const int j = r * SOR_RW + c;
        reinterpret_cast<float2 *>(dout)[(size_t)y * W + x] = make_float2(sdu[j], sdv[j]);
    }
}

__global__ void update_kernel(float *__restrict__ flow, float *__restrict__ d, long long n2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2;
         i += (long long)gridDim.x * blockDim.x) {
        flow[i] += d[i];
        d[i] = 0.f;
    }
}

unsigned grid_for(long long n, int num_sms) {
    long long b = (n + 255) / 256;
    const long long cap = (long long)num_sms * 8;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

// Scratch layout: warped image [P][C], coefficients [P][8], two update
// buffers [P][2]; every region starts on a 256-byte boundary (the blocked
// SOR reads coefficients as float4 and updates as float2).
static size_t rf_align(size_t b) { return (b + 255) / 256 * 256; }

size_t refine_scratch_bytes(int H, int W, int C) {
    const size_t P = (size_t)H * W;
    return rf_align(P * C * sizeof(float)) + rf_align(P * 8 * sizeof(float)) +
           2 * rf_align(P * 2 * sizeof(float));
}

cudaError_t launch_refine(const float *I1, const float *I2, int H, int W, int C, float *flow,
                          const RefineArgs &r, void *scratch, int num_sms, cudaStream_t stream) {
    const long long P = (long long)H * W;
    char *base = static_cast<char *>(scratch);
    float *I2w = reinterpret_cast<float *>(base);
    base += rf_align((size_t)P * C * sizeof(float));
    float *coef = reinterpret_cast<float *>(base);
    base += rf_align((size_t)P * 8 * sizeof(float));
    float *dbuf[2] = {reinterpret_cast<float *>(base),
                      reinterpret_cast<float *>(base + rf_align((size_t)P * 2 * sizeof(float)))};
    cudaError_t e = cudaMemsetAsync(dbuf[0], 0, sizeof(float) * 2 * P, stream);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(sor_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SOR_SMEM)) != cudaSuccess)
        return e;
    const unsigned gP = grid_for(P, num_sms);
    const unsigned g2 = grid_for(2 * P, num_sms);
    const dim3 gS((W + SOR_TX - 1) / SOR_TX, (H + SOR_TY - 1) / SOR_TY);
    Img i1{I1, H, W, C}, i2w{I2w, H, W, C};
    int cur = 0;   // the update buffer holding zeros / the latest update
    for (int it = 0; it < r.iterations; ++it) {
        warp_kernel<<<gP, 256, 0, stream>>>(I2, flow, H, W, C, I2w);
        coeff_kernel<<<gP, 256, 0, stream>>>(i1, i2w, flow, r, coef);
        // 2 * sor_iterations half-sweeps, SOR_H per launch (red first each
        // time, as SOR_H is even)
        for (int done = 0; done < 2 * r.sor_iterations; done += SOR_H) {
            const int nh = 2 * r.sor_iterations - done < SOR_H ? 2 * r.sor_iterations - done : SOR_H;
            sor_block_kernel<<<gS, 256, SOR_SMEM, stream>>>(flow, coef, H, W, r.omega, nh,
                                                            dbuf[cur], dbuf[cur ^ 1]);
            cur ^= 1;
        }
        update_kernel<<<g2, 256, 0, stream>>>(flow, dbuf[cur], 2 * P);   // adds, then zeroes
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace epic
