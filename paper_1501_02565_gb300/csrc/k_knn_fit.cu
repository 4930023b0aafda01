// Stage (c): for every match, its K nearest matches on G and the
// locally-weighted affine fit (Algorithm 1 steps 4-6, LA form; Eq. 2 with the
// kernel k = exp(-a D) of Eq. 1, restricted to N_K as in Sec. 3.2).
//
// One warp per match.  The search is Dijkstra on G from p_m under the key
// (graph distance, match index), so the K settled nodes are exactly the K
// smallest keys and ties at the K-th place go to the smaller index.  Per-warp
// shared memory holds
//   * an open-addressing table node -> tentative distance (bit 31 = settled),
//   * an unsorted frontier of packed keys (extract-min is a warp reduction,
//     an entry is pushed only when it strictly improves the node's distance;
//     stale entries are skipped or compacted away),
//   * the settled list (node, distance).
// Settling node v reads its adjacency row (one coalesced 8-byte load per
// lane); a newly pushed node's row is prefetched into L1 so that settling it
// later does not wait on L2.
//
// The fit uses centred coordinates x~ = p_n - p_m and fits the flow
// u = p' - p (the same least-squares problem as fitting p', Eq. 2, with
// A = I + B): 12 weighted sums, warp-reduced, then the 3x3 normal equations
// solved in float64.  The sums stay in float32 registers but are carried as
// unevaluated pairs hi + lo: every product w * t is split exactly with an FMA
// (TwoProduct) and every addition with TwoSum, so the accumulated sums keep
// about twice float32's precision.  Kernel weights span many decades when a
// neighbourhood crosses strong edges, and the normal matrix is then nearly
// singular along some direction; plain float32 sums lose that direction.  A degenerate fit (fewer than 3 neighbours or
// det M <= eps (tr M/3)^3) falls back to the Nadaraya-Watson estimate of
// Eq. 1 at p_m (kernel weights k), kept as a constant flow over the cell.
#include "epic_internal.cuh"

namespace epic {

namespace {

constexpr unsigned SETTLED = 0x80000000u;

__device__ __forceinline__ unsigned node_slot(unsigned u, int hs) {
    return (u * 0x9E3779B1u) >> 7 & (unsigned)(hs - 1);
}

// Slot holding node u (u is known to be present).
__device__ __forceinline__ unsigned find_node(const unsigned *hk, unsigned u, int hs) {
    unsigned s = node_slot(u, hs);
    for (int i = 0; i < hs; ++i) {
        if (hk[s] == u) return s;
        s = (s + 1) & (unsigned)(hs - 1);
    }
    return 0;  // unreachable for present nodes
}

// Compensated float32 accumulator: the value is hi + lo.
struct F2 {
    float hi, lo;
};

// Exact sum a + b = s + e (Knuth's TwoSum, no ordering assumption).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += a * b, with the product split exactly by an FMA.
__device__ __forceinline__ void acc_prod(F2 &acc, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    float s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}

// acc += v (v exact float)
__device__ __forceinline__ void acc_add(F2 &acc, float v) {
    float s, e;
    two_sum(acc.hi, v, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, e);
}

__device__ __forceinline__ F2 warp_sum(F2 v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, v.hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, v.lo, o);
        float s, e;
        two_sum(v.hi, oh, s, e);
        v.hi = s;
        v.lo = __fadd_rn(v.lo, __fadd_rn(ol, e));
    }
    return v;
}

__device__ __forceinline__ double to_d(F2 v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__global__ void __launch_bounds__(KNN_WARPS * 32) knn_fit_kernel(BatchArgs a) {
    const int warps = blockDim.x >> 5;
    extern __shared__ __align__(16) unsigned char smem[];
    RunState *st = a.state;
    if (get_status(st) != 0) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int HS = a.knn_hs, FS = a.knn_fs, KM = a.knn_kmax;
    const size_t per_warp = (size_t)FS * 8 + (size_t)HS * 8 + (size_t)KM * 8;
    unsigned char *base = smem + per_warp * wid;
    pkey_t *fk = reinterpret_cast<pkey_t *>(base);
    unsigned *hk = reinterpret_cast<unsigned *>(base + (size_t)FS * 8);
    unsigned *hv = hk + HS;
    unsigned *rn = hv + HS;
    float *rd = reinterpret_cast<float *>(rn + KM);
    const int md = a.max_degree;
    const unsigned lt_mask = (1u << lane) - 1u;

    for (int gm = blockIdx.x * warps + wid; gm < a.total_matches;
         gm += gridDim.x * warps) {
        const int pi = find_pair(a.match_base, a.npairs, gm);
        const PairDev &P = a.pairs[pi];
        const int m = gm - a.match_base[pi];
        const int K = P.K;
        const pkey_t *adj = P.adj;

        for (int i = lane; i < HS; i += 32) hk[i] = EMPTY32;
        __syncwarp();
        if (lane == 0) {
            unsigned s = node_slot((unsigned)m, HS);
            hk[s] = (unsigned)m;
            hv[s] = 0u;
            fk[0] = make_key(0.f, (unsigned)m);
        }
        __syncwarp();
        int fn = 1, cnt = 0;
        bool overflow = false;
        while (cnt < K && fn > 0 && !overflow) {
            // extract the smallest key
            pkey_t best = EMPTY64;
            int bpos = 0x7fffffff;
            for (int i = lane; i < fn; i += 32) {
                pkey_t k = fk[i];
                if (k < best) { best = k; bpos = i; }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                pkey_t ob = __shfl_xor_sync(0xffffffffu, best, o);
                int op = __shfl_xor_sync(0xffffffffu, bpos, o);
                if (ob < best || (ob == best && op < bpos)) { best = ob; bpos = op; }
            }
            __syncwarp();
            if (lane == 0) fk[bpos] = fk[fn - 1];
            fn -= 1;
            const unsigned v = key_label(best);
            const float d = key_dist(best);
            const unsigned sv = find_node(hk, v, HS);
            const unsigned hvv = hv[sv];
            __syncwarp();
            if ((hvv & SETTLED) || __uint_as_float(hvv) < d) continue;  // stale
            if (lane == 0) {
                hv[sv] = hvv | SETTLED;
                rn[cnt] = v;
                rd[cnt] = d;
            }
            ++cnt;
            if (cnt >= K) break;
            // relax v's edges
            for (int j0 = 0; j0 < md; j0 += 32) {
                const int j = j0 + lane;
                const pkey_t e = j < md ? __ldg(adj + (size_t)v * md + j) : EMPTY64;
                const bool has = e != EMPTY64;
                const unsigned u = (unsigned)e;
                const float nd = __fadd_rn(d, __uint_as_float((unsigned)(e >> 32)));
                bool push = false;
                if (has) {
                    unsigned s = node_slot(u, HS);
                    int probes = 0;
                    for (;;) {
                        const unsigned prev = atomicCAS(hk + s, EMPTY32, u);
                        if (prev == EMPTY32) {
                            hv[s] = __float_as_uint(nd);
                            push = true;
                            break;
                        }
                        if (prev == u) {
                            const unsigned cur = hv[s];
                            if (!(cur & SETTLED) && nd < __uint_as_float(cur)) {
                                hv[s] = __float_as_uint(nd);
                                push = true;
                            }
                            break;
                        }
                        s = (s + 1) & (unsigned)(HS - 1);
                        if (++probes >= HS) { overflow = true; break; }
                    }
                }
                unsigned bal = __ballot_sync(0xffffffffu, push);
                int np = __popc(bal);
                if (fn + np > FS) {
                    // drop stale entries (superseded or settled nodes)
                    __syncwarp();
                    int wpos = 0;
                    for (int b0 = 0; b0 < fn; b0 += 32) {
                        const int i = b0 + lane;
                        pkey_t k = 0;
                        bool keep = false;
                        if (i < fn) {
                            k = fk[i];
                            const unsigned cur = hv[find_node(hk, key_label(k), HS)];
                            keep = !(cur & SETTLED) && cur == (unsigned)(k >> 32);
                        }
                        const unsigned kb = __ballot_sync(0xffffffffu, keep);
                        __syncwarp();
                        if (keep) fk[wpos + __popc(kb & lt_mask)] = k;
                        wpos += __popc(kb);
                        __syncwarp();
                    }
                    fn = wpos;
                    if (fn + np > FS) overflow = true;
                }
                if (push && !overflow) {
                    fk[fn + __popc(bal & lt_mask)] = make_key(nd, u);
                    const pkey_t *row = adj + (size_t)u * md;
                    prefetch_l1(row);
                    if (md > 16) prefetch_l1(row + 16);
                }
                fn += np;
                overflow = __any_sync(0xffffffffu, overflow);
                __syncwarp();
                if (overflow) break;
                if (j0 + 32 < md && !__any_sync(0xffffffffu, has && lane == 31)) break;
            }
        }
        if (overflow) {
            if (lane == 0) set_status(st, EPIC_ERR_CAPACITY);
            cnt = 0;
        }
        __syncwarp();

        // locally-weighted affine fit over the cnt settled neighbours
        const float4 pm = __ldg(P.matches + m);
        F2 s[15];
#pragma unroll
        for (int i = 0; i < 15; ++i) s[i] = F2{0.f, 0.f};
        const float aa = P.a;
        for (int j = lane; j < cnt; j += 32) {
            const unsigned n = rn[j];
            const float dn = rd[j];
            const float4 q = __ldg(P.matches + n);
            const float k = expf(-__fmul_rn(aa, dn));
            const float w = a.weight_squared ? __fmul_rn(k, k) : k;
            // source coordinates are integral, so x~, y~ and their products
            // are exact; the flow u = x' - x is split exactly into uh + ul
            const float xt = __fsub_rn(q.x, pm.x), yt = __fsub_rn(q.y, pm.y);
            const float xx = __fmul_rn(xt, xt), xy = __fmul_rn(xt, yt), yy = __fmul_rn(yt, yt);
            float uh, ul, vh, vl;
            two_sum(q.z, -q.x, uh, ul);
            two_sum(q.w, -q.y, vh, vl);
            const float wx = __fmul_rn(w, xt), wy = __fmul_rn(w, yt);  // w * small integer
            acc_prod(s[0], w, xx);
            acc_prod(s[1], w, xy);
            acc_prod(s[2], w, xt);
            acc_prod(s[3], w, yy);
            acc_prod(s[4], w, yt);
            acc_add(s[5], w);
            acc_prod(s[6], wx, uh);  s[6].lo = __fmaf_rn(wx, ul, s[6].lo);
            acc_prod(s[7], wy, uh);  s[7].lo = __fmaf_rn(wy, ul, s[7].lo);
            acc_prod(s[8], w, uh);   s[8].lo = __fmaf_rn(w, ul, s[8].lo);
            acc_prod(s[9], wx, vh);  s[9].lo = __fmaf_rn(wx, vl, s[9].lo);
            acc_prod(s[10], wy, vh); s[10].lo = __fmaf_rn(wy, vl, s[10].lo);
            acc_prod(s[11], w, vh);  s[11].lo = __fmaf_rn(w, vl, s[11].lo);
            // Nadaraya-Watson sums (kernel k): k and k (p'_n - p_m)
            acc_add(s[12], k);
            float th, tl;
            two_sum(xt, uh, th, tl);
            acc_prod(s[13], k, th);
            s[13].lo = __fmaf_rn(k, __fadd_rn(tl, ul), s[13].lo);
            two_sum(yt, vh, th, tl);
            acc_prod(s[14], k, th);
            s[14].lo = __fmaf_rn(k, __fadd_rn(tl, vl), s[14].lo);
        }
        double S[15];
#pragma unroll
        for (int i = 0; i < 15; ++i) S[i] = to_d(warp_sum(s[i]));
        if (lane == 0) {
            const double M00 = S[0], M01 = S[1], M02 = S[2], M11 = S[3], M12 = S[4], M22 = S[5];
            // cofactors of the symmetric matrix M
            const double c00 = M11 * M22 - M12 * M12;
            const double c01 = M12 * M02 - M01 * M22;
            const double c02 = M01 * M12 - M11 * M02;
            const double c11 = M00 * M22 - M02 * M02;
            const double c12 = M01 * M02 - M00 * M12;
            const double c22 = M00 * M11 - M01 * M01;
            const double det = M00 * c00 + M01 * c01 + M02 * c02;
            const double tr3 = (M00 + M11 + M22) / 3.0;
            float4 r0, r1;
            int fb;
            if (cnt >= 3 && det > (double)a.fallback_eps * tr3 * tr3 * tr3) {
                const double ru0 = S[6], ru1 = S[7], ru2 = S[8];
                const double rv0 = S[9], rv1 = S[10], rv2 = S[11];
                const double id = 1.0 / det;
                const double bu0 = (c00 * ru0 + c01 * ru1 + c02 * ru2) * id;
                const double bu1 = (c01 * ru0 + c11 * ru1 + c12 * ru2) * id;
                const double bu2 = (c02 * ru0 + c12 * ru1 + c22 * ru2) * id;
                const double bv0 = (c00 * rv0 + c01 * rv1 + c02 * rv2) * id;
                const double bv1 = (c01 * rv0 + c11 * rv1 + c12 * rv2) * id;
                const double bv2 = (c02 * rv0 + c12 * rv1 + c22 * rv2) * id;
                r0 = make_float4((float)bu2, (float)bv2, (float)bu0, (float)bu1);
                r1 = make_float4((float)bv0, (float)bv1, pm.x, pm.y);
                fb = 0;
            } else {
                const double sk = S[12];
                r0 = make_float4((float)(S[13] / sk), (float)(S[14] / sk), 0.f, 0.f);
                r1 = make_float4(0.f, 0.f, pm.x, pm.y);
                fb = 1;
            }
            P.models[2 * (size_t)m] = r0;
            P.models[2 * (size_t)m + 1] = r1;
            P.fallback[m] = fb;
            if (P.knn_count) P.knn_count[m] = cnt;
        }
        if (P.knn_idx) {
            for (int j = lane; j < K; j += 32) {
                P.knn_idx[(size_t)m * K + j] = j < cnt ? (int)rn[j] : -1;
                P.knn_dist[(size_t)m * K + j] = j < cnt ? rd[j] : __int_as_float(0x7f800000);
            }
        }
        __syncwarp();
    }
}

int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace

void knn_table_sizes(int max_K, int *hs, int *fs) {
    *hs = next_pow2(max_K * 4 > 64 ? max_K * 4 : 64);
    *fs = next_pow2(max_K * 2 > 64 ? max_K * 2 : 64);
}

size_t knn_smem_per_warp(int max_K) {
    int hs, fs;
    knn_table_sizes(max_K, &hs, &fs);
    return (size_t)fs * 8 + (size_t)hs * 8 + (size_t)max_K * 8;
}

// Largest warps-per-CTA (<= KNN_WARPS) whose tables fit in shared memory;
// 0 if even one warp's tables do not fit.
int knn_warps_per_cta(int max_K, int smem_limit) {
    size_t pw = knn_smem_per_warp(max_K);
    int w = (int)(smem_limit / pw);
    return w > KNN_WARPS ? KNN_WARPS : w;
}

cudaError_t launch_knn_fit(const BatchArgs &a, const LaunchCfg &lc, int max_K) {
    int warps = knn_warps_per_cta(max_K, lc.smem_optin);
    if (warps < 1) return cudaErrorInvalidValue;
    size_t smem = knn_smem_per_warp(max_K) * warps;
    cudaError_t e = cudaFuncSetAttribute(
        knn_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, knn_fit_kernel,
                                                      warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    knn_fit_kernel<<<per_sm * lc.num_sms, warps * 32, smem, lc.stream>>>(a);
    return cudaGetLastError();
}

}  // namespace epic
