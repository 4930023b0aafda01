// Exact variant (Sec. 5.2, Table 2): every pixel takes its own K nearest
// matches under the exact distance and its own fit, instead of inheriting
// the model of its Voronoi cell (the approximation of Eq. 4).
//
//   keys_to_dist_kernel  turns a chunk of single-source relaxation results
//                        (one pseudo-pair per match, solved by the same
//                        relaxation kernel) into rows of D [N][P] float32;
//   exact_fit_kernel     one thread per pixel: scans D[m][p] over all m
//                        (coalesced across the warp's consecutive pixels),
//                        keeps the K smallest keys (distance, index) in a
//                        sorted list in shared memory, then fits Eq. 2
//                        centred at the pixel (FP64 sums and solve; the NW
//                        estimate of Eq. 1 when degenerate or requested) and
//                        writes the model's value at the pixel.  With the
//                        Euclidean distance D is not stored: the kernel
//                        computes |p - p_m| itself.
#include "epic_internal.cuh"

namespace epic {

namespace {

constexpr int EXACT_GROUP = 8;   // candidate distances loaded per group

__global__ void keys_to_dist_kernel(const pkey_t *keys, long long n, float *D) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        D[i] = key_dist(keys[i]);
}

// Seed offsets of the cap map (in key units): an upper bound of each
// match's K-th nearest graph distance, from the K-NN lists of an
// approximate run.  A graph distance is the cost of a real path (each edge
// weight is one), but summed in float from float-rounded weights, hence the
// relative and absolute margins.  Fewer than K neighbours: no bound.
__global__ void cap_seed_kernel(const float *knn_dist, const int *knn_count, int N, int K,
                                int ld, unsigned long long *init) {
    constexpr unsigned long long UNBOUNDED = 1ull << 40;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < N; m += gridDim.x * blockDim.x) {
        unsigned long long u = UNBOUNDED;
        if (knn_count[m] >= K) {
            const double d = (double)knn_dist[(size_t)m * ld + K - 1];
            if (d >= 0.0 && d < 256.0)
                u = min((unsigned long long)ceil(d * 2147483648.0 * (1.0 + 1.0 / 65536.0)) + 256ull,
                        UNBOUNDED);
        }
        init[m] = u;
    }
}

__device__ __forceinline__ unsigned long long dist_key(float d, unsigned m) {
    return ((unsigned long long)__float_as_uint(d) << 32) | m;
}

__global__ void __launch_bounds__(EXACT_THREADS) exact_fit_kernel(ExactArgs x) {
    extern __shared__ __align__(16) unsigned char smem[];
    // list entry j of thread t at j * blockDim.x + t (no bank conflicts)
    unsigned long long *list = reinterpret_cast<unsigned long long *>(smem);
    const int T = blockDim.x, t = threadIdx.x;
    const long long P = (long long)x.H * x.W;
    const long long p = blockIdx.x * (long long)T + t;
    if (p >= P) return;
    const int py = (int)(p / x.W), px = (int)(p - (long long)py * x.W);
    const int K = x.K;
    int cnt = 0;
    // candidates in groups of EXACT_GROUP: the group's distance loads are
    // all issued before any is used, so that many are in flight per thread
    for (int m0 = 0; m0 < x.N; m0 += EXACT_GROUP) {
        float dg[EXACT_GROUP];
#pragma unroll
        for (int u = 0; u < EXACT_GROUP; ++u) {
            const int m = m0 + u;
            float d = __int_as_float(0x7f800000);
            if (m < x.N) {
                if (x.D) {
                    d = __ldcs(x.D + (long long)m * P + p);
                } else {
                    const float4 q = __ldg(x.matches + m);
                    const float dx = __fsub_rn((float)px, floorf(q.x + 0.5f));
                    const float dy = __fsub_rn((float)py, floorf(q.y + 0.5f));
                    d = __fsqrt_rn(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)));
                }
            }
            dg[u] = d;
        }
#pragma unroll
        for (int u = 0; u < EXACT_GROUP; ++u) {
            const float d = dg[u];
            // an unreached distance (beyond the single-source run's cap, or
            // past the last match) cannot be among the K nearest: every pixel
            // has K matches within its cap
            if (!(d < __int_as_float(0x7f800000))) continue;
            const unsigned long long key = dist_key(d, (unsigned)(m0 + u));
            int j;
            if (cnt < K) {
                j = cnt - 1;
                ++cnt;
            } else if (key < list[(K - 1) * T + t]) {
                j = K - 2;
            } else {
                continue;
            }
            // insertion into the sorted list (ascending keys)
            while (j >= 0 && list[j * T + t] > key) {
                list[(j + 1) * T + t] = list[j * T + t];
                --j;
            }
            list[(j + 1) * T + t] = key;
        }
    }
    // fit centred at the pixel: rows (x~, y~, 1), x~ = x_n - x_p
    double M00 = 0, M01 = 0, M02 = 0, M11 = 0, M12 = 0, M22 = 0;
    double ru0 = 0, ru1 = 0, ru2 = 0, rv0 = 0, rv1 = 0, rv2 = 0;
    double sk = 0, sku = 0, skv = 0;
    for (int j = 0; j < cnt; ++j) {
        const unsigned long long key = list[j * T + t];
        const unsigned n = (unsigned)key;
        const double dn = (double)__uint_as_float((unsigned)(key >> 32));
        const float4 q = __ldg(x.matches + n);
        const double k = exp(-(double)x.a * dn);
        const double w = x.weight_squared ? k * k : k;
        const double xt = (double)q.x - px, yt = (double)q.y - py;
        const double u = (double)q.z - (double)q.x, v = (double)q.w - (double)q.y;
        M00 += w * xt * xt; M01 += w * xt * yt; M02 += w * xt;
        M11 += w * yt * yt; M12 += w * yt; M22 += w;
        ru0 += w * xt * u; ru1 += w * yt * u; ru2 += w * u;
        rv0 += w * xt * v; rv1 += w * yt * v; rv2 += w * v;
        sk += k; sku += k * u; skv += k * v;
        if (x.knn_idx) {
            x.knn_idx[p * K + j] = (int)n;
            x.knn_dist[p * K + j] = (float)dn;
        }
    }
    if (x.knn_idx) {
        for (int j = cnt; j < K; ++j) {
            x.knn_idx[p * K + j] = -1;
            x.knn_dist[p * K + j] = __int_as_float(0x7f800000);
        }
    }
    const double c00 = M11 * M22 - M12 * M12;
    const double c01 = M12 * M02 - M01 * M22;
    const double c02 = M01 * M12 - M11 * M02;
    const double c11 = M00 * M22 - M02 * M02;
    const double c12 = M01 * M02 - M00 * M12;
    const double c22 = M00 * M11 - M01 * M01;
    const double det = M00 * c00 + M01 * c01 + M02 * c02;
    const double tr3 = (M00 + M11 + M22) / 3.0;
    float fu, fv;
    int fb;
    if (x.estimator == 0 && cnt >= 3 && det > (double)x.fallback_eps * tr3 * tr3 * tr3) {
        // flow at the centre = the constant term of the fit
        const double id = 1.0 / det;
        fu = (float)((c02 * ru0 + c12 * ru1 + c22 * ru2) * id);
        fv = (float)((c02 * rv0 + c12 * rv1 + c22 * rv2) * id);
        fb = 0;
    } else {
        fu = (float)(sku / sk);
        fv = (float)(skv / sk);
        fb = 1;
    }
    x.flow[2 * p] = fu;
    x.flow[2 * p + 1] = fv;
    if (x.fallback) x.fallback[p] = fb;
}

}  // namespace

size_t exact_smem_bytes(int K) { return (size_t)K * EXACT_THREADS * sizeof(unsigned long long); }

cudaError_t launch_cap_seed(const float *knn_dist, const int *knn_count, int N, int K, int ld,
                            unsigned long long *init, cudaStream_t stream) {
    const int blocks = (N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024;
    cap_seed_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, stream>>>(knn_dist, knn_count, N, K, ld, init);
    return cudaGetLastError();
}

cudaError_t launch_keys_to_dist(const pkey_t *keys, long long n, float *D, cudaStream_t stream) {
    long long blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    keys_to_dist_kernel<<<(unsigned)blocks, 256, 0, stream>>>(keys, n, D);
    return cudaGetLastError();
}

cudaError_t launch_exact_fit(const ExactArgs &x, cudaStream_t stream) {
    const size_t smem = exact_smem_bytes(x.K);
    cudaError_t e = cudaFuncSetAttribute(exact_fit_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long P = (long long)x.H * x.W;
    const long long blocks = (P + EXACT_THREADS - 1) / EXACT_THREADS;
    exact_fit_kernel<<<(unsigned)blocks, EXACT_THREADS, smem, stream>>>(x);
    return cudaGetLastError();
}

}  // namespace epic
