// Stage (b): the match graph G (Sec. 3.4 "Approximated geodesic distance").
//
// Matches m and n are joined when their geodesic Voronoi cells touch, i.e.
// some 8-adjacent pixels p, q have L(p) = m, L(q) = n.  The edge weight is
// the geodesic distance from p_m to p_n restricted to the two cells, which
// is the minimum over touching pairs (p, q) of D(p) + step(p, q) + D(q): the
// shortest path from a seed to a pixel of its own cell stays in that cell,
// and a path inside the union crosses from one cell to the other at some
// touching pair.  Each candidate D(p) + step(p, q) + D(q) is summed exactly
// in the relaxation's fixed point and rounded once to float32.
//
// edges_kernel   every pixel looks at its four forward neighbours (right,
//                down-left, down, down-right: each unordered pixel pair once)
//                and forms (min label, max label, weight).  A work item is
//                a stack of relaxation tiles at least 32 rows high.
//                Candidates are merged per item (64 x 32 pixels hold only
//                tens of distinct label pairs): first over the pixel's four directions, then
//                across the lanes of a warp (match.any groups), then in a
//                shared-memory table with atomicMin on the weight; the tile's
//                unique entries are then inserted into the pair's global
//                open-addressing table.  Tiles are taken from a counter.  A match whose source pixel is owned
//                by a smaller index (a duplicate) is joined to the owner at
//                distance D = 0.
//                The insertion that creates an edge counts it in both
//                endpoints' degrees; every insertion lowers both endpoints'
//                lightest-edge weight.
// offsets_kernel one CTA per pair: exclusive scan of the degrees into the
//                CSR row offsets; the degree array becomes the fill cursor.
//                The pair's edge count is half the degree total (no shared
//                counter for the edges kernel to contend on).
// scatter_kernel every occupied slot appends (n, w) to row m and (m, w) to
//                row n of the CSR adjacency (order within a row unspecified;
//                the K-NN search does not depend on it).
// rowmin_kernel, bound_edge_kernel
//                per node the two lightest edges; then in every entry
//                (m -> n) the lightest edge at n other than (n, m).  The
//                K-NN search reads it with the entry (no dependent load)
//                for its step bound.
#include "epic_internal.cuh"

namespace epic {

namespace {

__device__ __forceinline__ unsigned hash_slot(pkey_t k, int cap) {
    unsigned long long h = k * 0x9E3779B97F4A7C15ull;
    return (unsigned)(h >> 32) & (unsigned)(cap - 1);
}

__device__ __forceinline__ void table_insert(const PairDev &P, pkey_t k,
                                             unsigned wbits, RunState *st) {
    unsigned s = hash_slot(k, P.hash_cap);
    const unsigned m = (unsigned)(k >> 32), n = (unsigned)k;
    for (int probe = 0; probe < P.hash_cap; ++probe) {
        pkey_t prev = atomicCAS(P.hkeys + s, EMPTY64, k);
        if (prev == EMPTY64 || prev == k) {
            atomicMin(P.hw + s, wbits);  // weights are >= 0: bit order = value order
            if (prev == EMPTY64) {       // a new edge
                atomicAdd(P.deg + m, 1);
                atomicAdd(P.deg + n, 1);
            }
            atomicMin(P.wmin + m, wbits);
            atomicMin(P.wmin + n, wbits);
            return;
        }
        s = (s + 1) & (unsigned)(P.hash_cap - 1);
    }
    set_status(st, EPIC_ERR_CAPACITY);
}

constexpr int TILE_TABLE = 1024;  // shared-memory slots per CTA (power of two)
constexpr int EDGE_ROWS = 32;     // a work item stacks relaxation tiles to this height

// Relaxation tiles a work item of the edge kernel stacks vertically: short
// tiles (the warp tiles are 64 x 16) would spend a larger share of the item
// on its halo and on taking the item.
__host__ __device__ __forceinline__ int edge_stack(int tile_h) {
    return tile_h >= EDGE_ROWS ? 1 : EDGE_ROWS / tile_h;
}

// Claim the shared-table slot of key k (or find it); -1 if the probe
// sequence is full.  A newly claimed slot is counted in *fill.
__device__ __forceinline__ int smem_claim(pkey_t *sk, pkey_t k, int *fill) {
    unsigned s = hash_slot(k, TILE_TABLE);
    for (int probe = 0; probe < 64; ++probe) {
        const pkey_t prev = atomicCAS(sk + s, EMPTY64, k);
        if (prev == EMPTY64) atomicAdd(fill, 1);
        if (prev == EMPTY64 || prev == k) return (int)s;
        s = (s + 1) & (TILE_TABLE - 1);
    }
    return -1;
}

// Insert one candidate per active lane.  Lanes holding the same label pair
// are grouped with one match.any; the group's lowest lane claims the slot in
// the shared table and every member lowers the slot's weight (or, if the
// table is full, inserts straight into the global table).
__device__ __forceinline__ void warp_insert(const PairDev &P, bool have, pkey_t k,
                                            unsigned wbits, pkey_t *sk, unsigned *sw,
                                            int *fill, RunState *st) {
    if (!__any_sync(0xffffffffu, have)) return;
    const unsigned lane = threadIdx.x & 31;
    const unsigned grp = __match_any_sync(0xffffffffu, have ? k : EMPTY64);
    const int leader = __ffs(grp) - 1;
    int slot = -1;
    if (have && lane == (unsigned)leader) slot = smem_claim(sk, k, fill);
    slot = __shfl_sync(0xffffffffu, slot, leader);
    if (have) {
        if (slot >= 0)
            atomicMin(sw + slot, wbits);
        else
            table_insert(P, k, wbits, st);
    }
}

__global__ void __launch_bounds__(EDGE_THREADS) edges_kernel(const BatchArgs *__restrict__ ap) {
    const BatchArgs a = *ap;
    RunState *st = a.state;
    if (get_status(st) != 0) return;
    __shared__ int s_tile, s_pair, s_local;
    __shared__ pkey_t sk[TILE_TABLE];
    __shared__ unsigned sw[TILE_TABLE];
    // the shared table collects the edges of consecutive tiles of one pair
    // and goes to the pair's global table when half full, when the next tile
    // belongs to another pair, and at the end
    __shared__ int s_fill, s_tab_pair;
    auto clear_table = [&]() {
        for (int i = threadIdx.x; i < TILE_TABLE; i += blockDim.x) {
            sk[i] = EMPTY64;
            sw[i] = 0xFFFFFFFFu;
        }
        if (threadIdx.x == 0) s_fill = 0;
        __syncthreads();
    };
    auto flush_table = [&](const PairDev &Q) {
        for (int i = threadIdx.x; i < TILE_TABLE; i += blockDim.x)
            if (sk[i] != EMPTY64) table_insert(Q, sk[i], sw[i], st);
        __syncthreads();
    };
    if (threadIdx.x == 0) s_tab_pair = -1;
    clear_table();
    // the tile's keys and half-costs plus the column on each side and the
    // row below (every forward neighbour), staged with coalesced loads that
    // are all in flight at once; cells outside the image hold KEY_INF
    extern __shared__ __align__(16) unsigned char edge_smem[];
    // tiles are handed out from a counter: their cost varies with the number
    // of cell boundaries they hold
    for (;;) {
        if (threadIdx.x == 0) {
            // an item starts at every edge_stack-th row of tiles; the tiles
            // in between belong to the item above them
            for (;;) {
                const int t = (int)atomicAdd(&st->edge_next, 1u);
                s_tile = t;
                if (t >= a.total_tiles) break;
                const int pi = find_pair(a.tile_base, a.npairs, t);
                const PairDev &Q = a.pairs[pi];
                const int lt = t - a.tile_base[pi];
                if ((lt / Q.tiles_x) % edge_stack(Q.tile_h) == 0) {
                    s_pair = pi;
                    s_local = lt;
                    break;
                }
            }
        }
        __syncthreads();
        if (s_tile >= a.total_tiles) break;
        // every thread takes the same decision from the shared values; they
        // change only after the barrier below
        if (s_tab_pair >= 0 && (s_tab_pair != s_pair || s_fill > TILE_TABLE / 2)) {
            flush_table(a.pairs[s_tab_pair]);
            clear_table();
        }
        __syncthreads();
        if (threadIdx.x == 0) s_tab_pair = s_pair;
        const PairDev &P = a.pairs[s_pair];
        // the pair's fields in registers (the table atomics below would
        // otherwise make every use a reload)
        const int TW = P.tile_w, TH = P.tile_h, TX = P.tiles_x, W = P.W, H = P.H;
        const unsigned NM = (unsigned)P.N;
        const pkey_t *keys = P.keys;
        const float *C = P.C;
        const int tx = s_local % TX, ty = s_local / TX;
        const int RH = edge_stack(TH) * TH;   // rows of the item
        const int npx = TW * RH;
        const int SC = TW + 2, SR = RH + 1;   // staged columns x0-1 .. x0+tw
        const int us = unit_shift(P);                      // the pair's distance unit
        const float unit = ldexpf(ONE_PER_UNIT, us);       // the distance of one unit
        pkey_t *skey = reinterpret_cast<pkey_t *>(edge_smem);
        unsigned *sh = reinterpret_cast<unsigned *>(skey + SC * SR);
        {
            // warp w stages rows w, w + 8, ...; its lanes take consecutive columns
            const int x0 = tx * TW - 1, y0 = ty * TH;
            const int nw = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
            bool bad = false;
            for (int r = wid; r < SR; r += nw) {
                const int gy = y0 + r;
                for (int c = lane; c < SC; c += 32) {
                    const int gx = x0 + c;
                    const bool in = gx >= 0 && gx < W && gy < H;
                    const size_t q = (size_t)gy * W + gx;
                    skey[r * SC + c] = in ? __ldg(keys + q) : KEY_INF;
                    sh[r * SC + c] = in ? half_cost_s(__ldg(C + q), us, &bad) : 0u;
                }
            }
        }
        __syncthreads();
        // tile widths are powers of two for the warp tiles (64): a shift
        const int tws = (TW & (TW - 1)) == 0 ? __ffs(TW) - 1 : -1;
        for (int i0 = 0; i0 < npx; i0 += blockDim.x) {  // warp-uniform trip count
            const int i = i0 + threadIdx.x;
            const int ly = tws >= 0 ? i >> tws : i / TW, lx = i - ly * TW;
            const int x = tx * TW + lx, y = ty * TH + ly;
            const bool act = i < npx && x < W && y < H;
            pkey_t kp = 0;
            unsigned hp = 0;
            if (act) {
                kp = skey[ly * SC + lx + 1];
                hp = sh[ly * SC + lx + 1];
            }
            // the four forward candidates of this pixel; a label pair seen in
            // an earlier direction is folded into that one (min weight), so
            // a pixel inserts each pair once
            pkey_t ck[4];
            unsigned cw[4];
            bool cv[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const int dx = d == 0 ? 1 : d == 1 ? -1 : d == 2 ? 0 : 1;
                const int dy = d == 0 ? 0 : 1;
                const int qx = x + dx, qy = y + dy;
                bool have = act && qx >= 0 && qx < W && qy < H;
                pkey_t k = 0;
                unsigned wb = 0;
                const int sq = (ly + dy) * SC + lx + 1 + dx;   // staged cell of q
                if (have) {
                    const pkey_t kq = skey[sq];
                    const unsigned lp = key_label(kp), lq = key_label(kq);
                    have = lp != lq;
                    if (have && (lp >= NM || lq >= NM ||
                                 !key_reached(kp) || !key_reached(kq))) {
                        // an unreached pixel (or a distance beyond the fixed-
                        // point range): the cost map was not in [0, C_MAX)
                        set_status(st, EPIC_ERR_INVALID);
                        have = false;
                    }
                    if (have) {
                        const unsigned hq = sh[sq];
                        const unsigned long long stp = (dx != 0 && dy != 0)
                                                           ? step_diag(hp, hq)
                                                           : step_axis(hp, hq);
                        // exact sum in fixed point, rounded once to float32
                        const unsigned long long units = key_dunits(kp) + stp + key_dunits(kq);
                        const float w = __fmul_rn(__ull2float_rn(units), unit);   // units_dist
                        k = lp < lq ? (((pkey_t)lp << 32) | lq) : (((pkey_t)lq << 32) | lp);
                        wb = __float_as_uint(w);
                    }
                }
#pragma unroll
                for (int j = 0; j < d; ++j) {
                    if (have && cv[j] && ck[j] == k) {
                        cw[j] = min(cw[j], wb);
                        have = false;
                    }
                }
                ck[d] = k;
                cw[d] = wb;
                cv[d] = have;
            }
            // this pixel's distinct candidates to the front (usually one or
            // two of the four directions), then one warp insertion round per
            // candidate rank that any lane holds
#pragma unroll
            for (int d = 1; d < 4; ++d) {
#pragma unroll
                for (int j = 0; j < d; ++j) {
                    if (!cv[j] && cv[d]) {
                        ck[j] = ck[d];
                        cw[j] = cw[d];
                        cv[j] = true;
                        cv[d] = false;
                    }
                }
            }
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                if (!__any_sync(0xffffffffu, cv[d])) break;
                warp_insert(P, cv[d], ck[d], cw[d], sk, sw, &s_fill, st);
            }
        }
        __syncthreads();
    }
    if (s_tab_pair >= 0) flush_table(a.pairs[s_tab_pair]);
    // duplicate source pixels: join an ownerless match to its pixel's owner
    for (int gm = blockIdx.x * blockDim.x + threadIdx.x; gm < a.total_matches;
         gm += gridDim.x * blockDim.x) {
        const int p = find_pair(a.match_base, a.npairs, gm);
        const PairDev &P = a.pairs[p];
        const int m = gm - a.match_base[p];
        const float4 mt = __ldg(P.matches + m);
        const int x = (int)floorf(mt.x + 0.5f), y = (int)floorf(mt.y + 0.5f);
        const pkey_t kp = __ldg(P.keys + (size_t)y * P.W + x);
        const unsigned l = key_label(kp);
        if (l != (unsigned)m && l < (unsigned)P.N) {
            const unsigned lo = min(l, (unsigned)m), hi = max(l, (unsigned)m);
            table_insert(P, ((pkey_t)lo << 32) | hi,
                         __float_as_uint(units_dist(key_dunits(kp), unit_shift(P))), st);
        }
    }
}

// Exclusive scan of v[0..n) into out[0..n] (out[n] = total) and v[i] =
// out[i], by one CTA; returns the largest v[i] to thread 0.
__device__ int block_offsets(int *v, int *out, int n) {
    __shared__ int warp_sums[32];
    __shared__ int carry, vmax;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) { carry = 0; vmax = 0; }
    __syncthreads();
    int mx = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + tid;
        const int x = i < n ? v[i] : 0;
        mx = max(mx, x);
        int sc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, sc, o);
            if (lane >= o) sc += t;
        }
        if (lane == 31) warp_sums[wid] = sc;
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
        const int excl = carry + sc - x + (wid > 0 ? warp_sums[wid - 1] : 0);
        if (i < n) {
            out[i] = excl;
            v[i] = excl;   // the fill cursor of row i
        }
        __syncthreads();
        if (tid == blockDim.x - 1) carry = excl + x;
        __syncthreads();
    }
    atomicMax(&vmax, mx);
    __syncthreads();
    if (tid == 0) out[n] = carry;
    return vmax;
}

__global__ void __launch_bounds__(1024) offsets_kernel(const BatchArgs *__restrict__ ap) {
    const BatchArgs a = *ap;
    if (get_status(a.state) != 0) return;
    for (int p = blockIdx.x; p < a.npairs; p += gridDim.x) {
        const PairDev &P = a.pairs[p];
        const int mx = block_offsets(P.deg, P.row, P.N);
        if (threadIdx.x == 0) {
            P.info[0] = P.row[P.N] / 2;   // edges: every edge is in two rows
            P.info[1] = mx;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) scatter_kernel(const BatchArgs *__restrict__ ap) {
    const BatchArgs a = *ap;
    RunState *st = a.state;
    if (get_status(st) != 0) return;
    for (int gs = blockIdx.x * blockDim.x + threadIdx.x; gs < a.total_hash;
         gs += gridDim.x * blockDim.x) {
        const int p = find_pair(a.hash_base, a.npairs, gs);
        const PairDev &P = a.pairs[p];
        const int s = gs - a.hash_base[p];
        const pkey_t k = P.hkeys[s];
        if (k == EMPTY64) continue;
        const unsigned m = (unsigned)(k >> 32), n = (unsigned)k;
        if (m >= (unsigned)P.N || n >= (unsigned)P.N) {
            set_status(st, EPIC_ERR_INVALID);
            continue;
        }
        const unsigned wb = P.hw[s];
        P.adj[atomicAdd(P.deg + m, 1)] = make_uint4(n, wb, 0u, m);
        P.adj[atomicAdd(P.deg + n, 1)] = make_uint4(m, wb, 0u, n);
    }
}

// Per node: the two lightest edge weights (the second is +inf below two
// edges) and the other end of the lightest.
__global__ void __launch_bounds__(256) rowmin_kernel(const BatchArgs *__restrict__ ap) {
    const BatchArgs a = *ap;
    if (get_status(a.state) != 0) return;
    for (int gm = blockIdx.x * blockDim.x + threadIdx.x; gm < a.total_matches;
         gm += gridDim.x * blockDim.x) {
        const int pi = find_pair(a.match_base, a.npairs, gm);
        const PairDev &P = a.pairs[pi];
        const int m = gm - a.match_base[pi];
        unsigned w1 = 0x7F800000u, w2 = 0x7F800000u;
        int n1 = -1;
        for (int j = P.row[m], e = P.row[m + 1]; j < e; ++j) {
            const uint4 ed = P.adj[j];
            if (ed.y < w1) {
                w2 = w1;
                w1 = ed.y;
                n1 = (int)ed.x;
            } else if (ed.y < w2) {
                w2 = ed.y;
            }
        }
        P.wmin2[m] = w2;
        P.wnear[m] = n1;
    }
}

// Per CSR entry (m -> n): the lightest edge at n other than the one back to
// m, which is what a K-NN search that reaches n from m adds to n's distance
// for its step bound (see k_knn_fit.cu).  A thread per entry slot of the
// pairs' adjacency arrays (2 x hash_cap each, the used ones first); the
// entry carries its row node m.
__global__ void __launch_bounds__(256) bound_edge_kernel(const BatchArgs *__restrict__ ap) {
    const BatchArgs a = *ap;
    if (get_status(a.state) != 0) return;
    for (long long gs = blockIdx.x * (long long)blockDim.x + threadIdx.x;
         gs < 2LL * a.total_hash; gs += (long long)gridDim.x * blockDim.x) {
        const int pi = find_pair(a.hash_base, a.npairs, (int)(gs >> 1));
        const PairDev &P = a.pairs[pi];
        const int j = (int)(gs - 2LL * a.hash_base[pi]);
        if (j >= P.row[P.N]) continue;
        const uint4 ed = P.adj[j];
        const int n = (int)ed.x, m = (int)ed.w;
        P.adj[j].z = P.wnear[n] == m ? P.wmin2[n] : P.wmin[n];
    }
}

__global__ void split_kernel(const pkey_t *keys, int P, int *labels, float *dist,
                             const PairDev *pair_dev) {
    const int us = unit_shift(*pair_dev);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        pkey_t k = keys[i];
        if (labels) labels[i] = (int)key_label(k);
        if (dist) dist[i] = key_reached(k) ? units_dist(key_dunits(k), us)
                                           : __int_as_float(0x7f800000);
    }
}

__global__ void collect_kernel(const pkey_t *hkeys, const unsigned *hw, int cap_slots,
                               int *em, int *en, float *ew, int cap, int *count) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < cap_slots;
         s += gridDim.x * blockDim.x) {
        pkey_t k = hkeys[s];
        if (k == EMPTY64) continue;
        int i = atomicAdd(count, 1);
        if (i < cap) {
            em[i] = (int)(k >> 32);
            en[i] = (int)(unsigned)k;
            ew[i] = __uint_as_float(hw[s]);
        }
    }
}

}  // namespace

size_t edges_smem_bytes(int max_tile_w, int max_tile_h) {
    // stacked tiles are at most EDGE_ROWS rows high (a taller tile is one item)
    const int rows = max_tile_h > EDGE_ROWS ? max_tile_h : EDGE_ROWS;
    return (size_t)(max_tile_w + 2) * (rows + 1) * (sizeof(pkey_t) + sizeof(unsigned));
}

cudaError_t launch_edges(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc,
                         int max_tile_w, int max_tile_h) {
    (void)a;
    const size_t smem = edges_smem_bytes(max_tile_w, max_tile_h);
    cudaError_t e = cudaFuncSetAttribute(edges_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // one resident wave: every CTA keeps taking tiles until none are left
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edges_kernel, EDGE_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    edges_kernel<<<lc.num_sms * per_sm, EDGE_THREADS, smem, lc.stream>>>(dev);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc) {
    int g = a.npairs < lc.num_sms ? a.npairs : lc.num_sms;
    offsets_kernel<<<g < 1 ? 1 : g, 1024, 0, lc.stream>>>(dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scatter_kernel<<<lc.num_sms * 4, 256, 0, lc.stream>>>(dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    rowmin_kernel<<<lc.num_sms * 4, 256, 0, lc.stream>>>(dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    bound_edge_kernel<<<lc.num_sms * 4, 256, 0, lc.stream>>>(dev);
    return cudaGetLastError();
}

cudaError_t launch_split_keys(const PairDev *P, const PairDev *pair_dev, int *labels,
                              float *dist, cudaStream_t stream) {
    int n = P->H * P->W;
    split_kernel<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, stream>>>(
        P->keys, n, labels, dist, pair_dev);
    return cudaGetLastError();
}

cudaError_t launch_collect_edges(const PairDev *P, int *em, int *en, float *ew,
                                 int cap, int *count, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    int blocks = (P->hash_cap + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    collect_kernel<<<blocks, 256, 0, stream>>>(P->hkeys, P->hw, P->hash_cap, em, en,
                                               ew, cap, count);
    return cudaGetLastError();
}

}  // namespace epic
