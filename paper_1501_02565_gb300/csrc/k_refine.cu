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
//   sor_kernel     one half-sweep (one colour) of point-coupled SOR: the
//                  2x2 system of (du, dv) at a pixel is solved exactly from
//                  the current neighbours and over-relaxed;
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

// One half-sweep: every pixel of `colour` ((x + y) & 1 == colour).  Thread t
// of row y takes column 2 t + ((y + colour) & 1), so consecutive threads
// take consecutive pixels of that colour.
__global__ void sor_kernel(const float *__restrict__ flow, const float *__restrict__ coef, int H,
                           int W, float omega, int colour, float *__restrict__ d) {
    const int half = (W + 1) / 2;
    const long long n = (long long)H * half;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / half);
        const int x = 2 * (int)(i - (long long)y * half) + ((y + colour) & 1);
        if (x >= W) continue;
        const size_t p = (size_t)y * W + x;
        const float *cp = coef + p * 8;
        const float phip = cp[5];
        const float up = flow[2 * p], vp = flow[2 * p + 1];
        float S = 0.f, r1 = 0.f, r2 = 0.f;
        auto nb = [&](size_t q) {
            const float s = 0.5f * (phip + coef[q * 8 + 5]);
            S += s;
            r1 += s * (flow[2 * q] + d[2 * q] - up);
            r2 += s * (flow[2 * q + 1] + d[2 * q + 1] - vp);
        };
        if (x + 1 < W) nb(p + 1);
        if (x > 0) nb(p - 1);
        if (y + 1 < H) nb(p + W);
        if (y > 0) nb(p - W);
        r1 -= cp[3];
        r2 -= cp[4];
        const float a = cp[0] + S, b = cp[1], dd = cp[2] + S;
        const float det = a * dd - b * b;
        if (!(det > 0.f)) continue;
        const float nu = (dd * r1 - b * r2) / det, nv = (a * r2 - b * r1) / det;
        d[2 * p] = (1.f - omega) * d[2 * p] + omega * nu;
        d[2 * p + 1] = (1.f - omega) * d[2 * p + 1] + omega * nv;
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

size_t refine_scratch_bytes(int H, int W, int C) {
    const size_t P = (size_t)H * W;
    return P * C * sizeof(float) + P * 8 * sizeof(float) + P * 2 * sizeof(float);
}

cudaError_t launch_refine(const float *I1, const float *I2, int H, int W, int C, float *flow,
                          const RefineArgs &r, void *scratch, int num_sms, cudaStream_t stream) {
    const long long P = (long long)H * W;
    float *I2w = static_cast<float *>(scratch);
    float *coef = I2w + P * C;
    float *d = coef + P * 8;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(float) * 2 * P, stream);
    if (e != cudaSuccess) return e;
    const unsigned gP = grid_for(P, num_sms);
    const unsigned gH = grid_for((long long)H * ((W + 1) / 2), num_sms);
    const unsigned g2 = grid_for(2 * P, num_sms);
    Img i1{I1, H, W, C}, i2w{I2w, H, W, C};
    for (int it = 0; it < r.iterations; ++it) {
        warp_kernel<<<gP, 256, 0, stream>>>(I2, flow, H, W, C, I2w);
        coeff_kernel<<<gP, 256, 0, stream>>>(i1, i2w, flow, r, coef);
        for (int s = 0; s < r.sor_iterations; ++s) {
            sor_kernel<<<gH, 256, 0, stream>>>(flow, coef, H, W, r.omega, 0, d);
            sor_kernel<<<gH, 256, 0, stream>>>(flow, coef, H, W, r.omega, 1, d);
        }
        update_kernel<<<g2, 256, 0, stream>>>(flow, d, 2 * P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace epic
