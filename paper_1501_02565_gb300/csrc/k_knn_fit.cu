// Stage (c): for every match, its K nearest matches on G and the
// locally-weighted affine fit (Algorithm 1 steps 4-6, LA form; Eq. 2 with the
// kernel k = exp(-a D) of Eq. 1, restricted to N_K as in Sec. 3.2).
//
// One warp per match.  The search is Dijkstra on G from p_m under the key
// (graph distance, match index), run in batches: a step settles every
// frontier node u whose tentative distance is below
//     B = min over frontier entries v of (t(v) + w_x(v)),
// where w_x(v) is the lightest edge at v other than the edge to the settled
// node whose relaxation gave v its current distance (for the source, its
// lightest edge), plus the smallest key, always.  A path that can still
// shorten a node leaves the settled set through some frontier node v and
// then an edge of v to an unsettled node, which is not the edge back to v's
// settled parent, so it costs at least t(v) + w_x(v) >= B; hence no
// frontier node below B can be shortened, every node settled later ends at
// a distance >= B, and a batch sorted by key extends the settled list in
// exactly the order sequential Dijkstra would produce, ties at the K-th
// place going to the smaller index.  A batch is usually several nodes, so a
// match needs ~5x fewer steps than one-node-at-a-time settling; excluding
// the parent edge from the bound saves another ~13 % of the steps.
// Per-warp shared memory holds
//   * the frontier: packed keys (t bits << 32 | node), their table slots and
//     t + w_x, rebuilt every step so that only current entries survive,
//   * an open-addressing table node -> tentative distance (0 = settled):
//     a lane claims a node's slot with compare-and-swap and lowers its
//     distance with atomicMin, so several lanes may relax into one node,
//   * the settled list (node, distance, start of its batch).
// The main pass sizes these tables for the searches seen on optical-flow
// match graphs (about 1.5 K nodes touched) so that four CTAs of eight warps
// share an SM; a search that outgrows them is queued and run again by a
// second launch with one warp per CTA and tables ~20x larger, so no
// neighbourhood shape fails.
// Batches are appended in frontier order; only the batch that crosses K is
// sorted (warp bitonic network) so that exactly the K smallest keys are
// kept, and every batch of the finished list is sorted before the fit.  All
// edges of all batch nodes are relaxed in one pass: lanes take (node, edge)
// pairs found from a warp prefix sum of the batch nodes' degrees (CSR row
// lengths).  A newly pushed node's w_x comes with the adjacency entry
// (precomputed per CSR entry by the graph stage), since the step's bound is
// kept as a running minimum over the entries pushed and kept (no separate
// pass over the frontier).  The step's smallest
// key and bound are then two 32-bit warp reductions (redux.sync).
//
// The fit uses centred coordinates x~ = p_n - p_m and fits the flow
// u = p' - p (the same least-squares problem as fitting p', Eq. 2, with
// A = I + B): 12 weighted sums, warp-reduced by a transposed reduction that
// leaves each sum on two lanes, then the 3x3 normal equations solved in
// float64 by cofactors, spread over the lanes of the warp.  The
// sums stay in float32 registers but are carried as unevaluated pairs hi + lo: every product w * t is split exactly with an FMA
// (TwoProduct) and every addition with TwoSum, so the accumulated sums keep
// about twice float32's precision.  Kernel weights span many decades when a
// neighbourhood crosses strong edges, and the normal matrix is then nearly
// singular along some direction; plain float32 sums lose that direction.  A
// degenerate fit (fewer than 3 neighbours or det M <= eps (tr M/3)^3) falls back to the Nadaraya-Watson estimate of
// Eq. 1 at p_m (kernel weights k), kept as a constant flow over the cell.
#include "epic_internal.cuh"

#include <algorithm>

namespace epic {

namespace {

// Node-table distance word: the float bits of the tentative distance plus
// one while the node is unsettled (+inf: 0x7F800001), 0 once it is settled,
// so that one atomicMin both lowers a tentative distance and leaves a
// settled node alone.
constexpr unsigned SETTLED = 0u;
constexpr unsigned DIST_INF = 0x7F800001u;
__device__ __forceinline__ unsigned dist_word(unsigned dist_bits) { return dist_bits + 1u; }

// Search key on G: float32 bits of the graph distance (non-negative, so the
// bit pattern orders like the value) above the 32-bit node index.
__device__ __forceinline__ pkey_t make_key(float d, unsigned node) {
    return ((pkey_t)__float_as_uint(d) << 32) | node;
}
__device__ __forceinline__ float key_dist(pkey_t k) {
    return __uint_as_float((unsigned)(k >> 32));
}
__device__ __forceinline__ unsigned key_label(pkey_t k) { return (unsigned)k; }

__device__ __forceinline__ unsigned node_slot(unsigned u, int hs) {
    return __umulhi(u * 0x9E3779B1u, (unsigned)hs);   // any table size
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

__device__ __forceinline__ double to_d(F2 v) { return (double)v.hi + (double)v.lo; }

// One frontier entry: packed key (t bits << 32 | node), its node-table slot
// and t + w_x, moved as one 16-byte access.
struct __align__(16) FEnt {
    pkey_t k;
    unsigned sl;
    float tw;
};

// Per-warp tables: frontier [fs], node table [hs] x 2 words, settled list
// [km] x (node, distance) and batch starts [km] x 2 bytes; 16-byte multiple.
__host__ __device__ __forceinline__ size_t knn_fixed_bytes(int km) {
    return ((size_t)km * 8 + (((size_t)km * 2 + 7) & ~(size_t)7) + 15) & ~(size_t)15;
}
__host__ __device__ __forceinline__ size_t knn_warp_bytes(int hs, int fs, int km) {
    return (size_t)fs * sizeof(FEnt) + (((size_t)hs * 8 + 15) & ~(size_t)15) + knn_fixed_bytes(km);
}

// Sort the settled list (node, distance) by key (distance, node) in place.
// Batches were appended in key order (every key of a batch is below the
// bound B of its step, every later key at least B), so an entry's sorted
// position is its batch's start plus its rank within the batch; bs[i] holds
// the start of entry i's batch.  `scratch` (>= n keys) is workspace; one warp.
__device__ void sort_settled(unsigned *rn, float *rd, const unsigned short *bs, int n,
                             pkey_t *scratch, int lane) {
    for (int i = lane; i < n; i += 32) {
        const int b = bs[i];
        const pkey_t ki = make_key(rd[i], rn[i]);
        int r = 0;
        for (int j = b; j < n && bs[j] == b; ++j) r += make_key(rd[j], rn[j]) < ki;
        scratch[b + r] = ki;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        rn[i] = key_label(scratch[i]);
        rd[i] = key_dist(scratch[i]);
    }
    __syncwarp();
}

// HS, FS: this launch's table sizes.  RETRY = false: the main pass (small
// tables, several CTAs per SM; a match that outgrows them is queued); true:
// the pass over the queued matches (large tables, one warp per CTA), which
// returns at once when nothing was queued.
template <bool RETRY>
__global__ void __launch_bounds__(KNN_WARPS * 32, 4)
    knn_fit_kernel(const BatchArgs *__restrict__ ap, int HS, int FS) {
    if (RETRY && *(volatile const unsigned *)&ap->state->knn_overflow == 0u) return;
    const BatchArgs a = *ap;
    extern __shared__ __align__(16) unsigned char smem[];
    RunState *st = a.state;
    if (get_status(st) != 0) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int KM = a.knn_kmax;
    const size_t per_warp = knn_warp_bytes(HS, FS, KM);
    unsigned char *base = smem + per_warp * wid;
    FEnt *fe = reinterpret_cast<FEnt *>(base);              // frontier
    unsigned *hk = reinterpret_cast<unsigned *>(fe + FS);   // node table: node
    unsigned *hv = hk + HS;                                 // distance word (0 = settled)
    unsigned *rn = reinterpret_cast<unsigned *>(
        reinterpret_cast<unsigned char *>(hk) + ((((size_t)HS * 8) + 15) & ~(size_t)15));
    float *rd = reinterpret_cast<float *>(rn + KM);
    // batch start of each settled entry (K stays far below 65536: the tables of one
    // warp must fit in shared memory)
    unsigned short *bs = reinterpret_cast<unsigned short *>(rd + KM);
    const unsigned lt_mask = (1u << lane) - 1u;

    // matches are handed out one at a time from a counter: search costs
    // vary with the neighbourhood, and a static split leaves a long tail
    for (;;) {
        int gm = 0;
        if (RETRY) {
            const unsigned nq = min(*(volatile unsigned *)&st->knn_overflow, (unsigned)a.total_matches);
            unsigned q = 0;
            if (lane == 0) q = atomicAdd(&st->knn_retry, 1u);
            q = __shfl_sync(0xffffffffu, q, 0);
            if (q >= nq) break;
            gm = a.knn_retry_list[q];
        } else {
            if (lane == 0) gm = (int)atomicAdd(&st->knn_next, 1u);
            gm = __shfl_sync(0xffffffffu, gm, 0);
            if (gm >= a.total_matches) break;
        }
        const int pi = find_pair(a.match_base, a.npairs, gm);
        const PairDev &P = a.pairs[pi];
        const int m = gm - a.match_base[pi];
        const int K = P.K;
        const uint4 *adj = P.adj;
        const unsigned *wmin = P.wmin;

        for (int i = lane; i < HS; i += 32) {
            hk[i] = EMPTY32;
            hv[i] = DIST_INF;
        }
        __syncwarp();
        // each lane's running minimum of the keys and of t + w_x over the
        // frontier entries it kept or pushed since the last step: the step's
        // smallest key and bound B are their warp minima.  Stale entries
        // (a node pushed again with a smaller key) only add larger values
        // than the node's current entry, so the minima are exact.
        pkey_t rk = EMPTY64;
        float rb = __int_as_float(0x7f800000);
        if (lane == 0) {
            const unsigned s0 = node_slot((unsigned)m, HS);
            hk[s0] = (unsigned)m;
            hv[s0] = dist_word(0u);
            rk = make_key(0.f, (unsigned)m);
            rb = __fadd_rn(0.f, __uint_as_float(__ldg(wmin + m)));
            fe[0] = FEnt{rk, s0, rb};
        }
        __syncwarp();
        int fn = 1, cnt = 0;
        bool overflow = false;
        while (cnt < K) {
            // (1) smallest current key and the batch bound B, as warp
            //     reductions of 32-bit words: distances are non-negative, so
            //     their float bits order like the values (+inf included)
            const unsigned kd = __reduce_min_sync(0xffffffffu, (unsigned)(rk >> 32));
            const unsigned kn =
                __reduce_min_sync(0xffffffffu, (unsigned)(rk >> 32) == kd ? (unsigned)rk : EMPTY32);
            const pkey_t kmin = ((pkey_t)kd << 32) | kn;
            const float bound = __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(rb)));
            if (kmin == EMPTY64) break;  // component exhausted
            rk = EMPTY64;
            rb = __int_as_float(0x7f800000);
            // (2) the batch: current entries below the bound (and the
            //     smallest).  A batch that reaches K is finished by sorting it
            //     in lanes; one reaching K with more than a warp of entries is
            //     cut to the smallest key alone.
            // (fn counts every frontier entry, an upper bound on the batch:
            // while cnt + fn < K the batch cannot reach K and is not counted)
            int nwin = 0;
            for (int b0 = 0; cnt + fn >= K && b0 < fn; b0 += 32) {
                const int i = b0 + lane;
                bool inb = false;
                if (i < fn) {
                    const FEnt f = fe[i];
                    const pkey_t k = f.k;
                    const unsigned cur = hv[f.sl];
                    inb = cur == dist_word((unsigned)(k >> 32)) &&
                          (key_dist(k) < bound || k == kmin);
                }
                nwin += __popc(__ballot_sync(0xffffffffu, inb));
            }
            const bool final_batch = cnt + nwin >= K && nwin <= 32;
            const bool single = cnt + nwin >= K && nwin > 32;
            // (3) partition: kept entries are compacted to the front (writes
            //     never pass reads); batch entries are settled into the list
            //     or, for the final batch, handed to lanes
            int wpos = 0, nb = 0;
            pkey_t bk = EMPTY64;
            for (int b0 = 0; b0 < fn; b0 += 32) {
                const int i = b0 + lane;
                pkey_t k = EMPTY64;
                unsigned sl = 0;
                float tw = 0.f;
                bool valid = false;
                if (i < fn) {
                    const FEnt f = fe[i];
                    k = f.k;
                    sl = f.sl;
                    tw = f.tw;
                    const unsigned cur = hv[sl];
                    valid = cur == dist_word((unsigned)(k >> 32));
                }
                const bool inb = valid && (single ? k == kmin
                                                  : (key_dist(k) < bound || k == kmin));
                const bool keep = valid && !inb;
                const unsigned kb = __ballot_sync(0xffffffffu, keep);
                const unsigned bb = __ballot_sync(0xffffffffu, inb);
                __syncwarp();
                if (keep) {
                    const int p = wpos + __popc(kb & lt_mask);
                    fe[p] = FEnt{k, sl, tw};
                    rk = k < rk ? k : rk;
                    rb = fminf(rb, tw);
                }
                if (final_batch) {
                    unsigned rem = bb;
                    while (rem) {
                        const int src = __ffs(rem) - 1;
                        rem &= rem - 1;
                        const pkey_t xk = __shfl_sync(0xffffffffu, k, src);
                        if (lane == nb) bk = xk;
                        ++nb;
                    }
                } else {
                    if (inb) {
                        const int p = cnt + nb + __popc(bb & lt_mask);
                        hv[sl] = SETTLED;
                        rn[p] = key_label(k);
                        rd[p] = key_dist(k);
                        bs[p] = (unsigned short)cnt;
                    }
                    nb += __popc(bb);
                }
                wpos += __popc(kb);
                __syncwarp();
            }
            fn = wpos;
            if (final_batch) {
                // sort the final batch by key across lanes (bitonic) and keep
                // the smallest K - cnt
#pragma unroll
                for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
                    for (int j = kk >> 1; j > 0; j >>= 1) {
                        const pkey_t ok = __shfl_xor_sync(0xffffffffu, bk, j);
                        const bool asc = (lane & kk) == 0;
                        const bool lower = (lane & j) == 0;
                        if ((lower == asc) ? (ok < bk) : (ok > bk)) bk = ok;
                    }
                }
                if (cnt + lane < K) {
                    rn[cnt + lane] = key_label(bk);
                    rd[cnt + lane] = key_dist(bk);
                    bs[cnt + lane] = (unsigned short)cnt;
                }
                cnt = K;
                __syncwarp();
                break;
            }
            const int c0 = cnt;
            cnt += nb;
            __syncwarp();
            if (cnt >= K) break;
            // (4) relax every edge of every batch node in one pass
            for (int b0 = 0; b0 < nb && !overflow; b0 += 32) {
                const int bi = b0 + lane;
                const bool hb = bi < nb;
                const pkey_t vk = hb ? make_key(rd[c0 + bi], rn[c0 + bi]) : EMPTY64;
                // CSR row of the batch node: its first entry and its degree
                int rbeg = 0, dg = 0;
                if (hb) {
                    const unsigned v = key_label(vk);
                    rbeg = __ldg(P.row + v);
                    dg = __ldg(P.row + v + 1) - rbeg;
                }
                // the chunk's batch nodes sit in lanes [0, nbc): the scan and
                // the owner search need only ceil(log2 nbc) levels (batches
                // average ~5 nodes)
                const int nbc = min(nb - b0, 32);
                int top = 1;
                while (top < nbc) top <<= 1;
                int incl = dg;
                for (int o = 1; o < top; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                const int excl = incl - dg;
                const int total = __shfl_sync(0xffffffffu, incl, nbc - 1);
                for (int e0 = 0; e0 < total; e0 += 32) {
                    const int e = e0 + lane;
                    // owner: the last lane whose edge range starts at or before e
                    int owner = 0;
                    for (int stp = top >> 1; stp; stp >>= 1) {
                        const int cand = owner + stp;
                        const int ex = __shfl_sync(0xffffffffu, excl, cand & 31);
                        if (cand < nbc && ex <= e) owner = cand;
                    }
                    const pkey_t ok = __shfl_sync(0xffffffffu, vk, owner);
                    const int oex = __shfl_sync(0xffffffffu, excl, owner);
                    const int obeg = __shfl_sync(0xffffffffu, rbeg, owner);
                    const bool act = e < total;
                    bool push = false;
                    unsigned slot = 0, u = 0, uw = 0;
                    float nd = 0.f;
                    if (act) {
                        const uint4 ed = __ldg(adj + obeg + (e - oex));
                        u = ed.x;
                        uw = ed.z;
                        nd = __fadd_rn(key_dist(ok), __uint_as_float(ed.y));
                        unsigned sl = node_slot(u, HS);
                        int probes = 0;
                        for (;;) {
                            const unsigned prev = atomicCAS(hk + sl, EMPTY32, u);
                            if (prev == EMPTY32 || prev == u) break;
                            sl = sl + 1 == (unsigned)HS ? 0u : sl + 1;
                            if (++probes >= HS) { overflow = true; break; }
                        }
                        if (!overflow) {
                            // a settled node (word 0) is never lowered
                            const unsigned w = dist_word(__float_as_uint(nd));
                            push = w < atomicMin(hv + sl, w);
                        }
                        slot = sl;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, push);
                    const int np = __popc(bal);
                    if (fn + np > FS) {
                        // drop entries superseded since this step's rebuild
                        __syncwarp();
                        int w2 = 0;
                        for (int q0 = 0; q0 < fn; q0 += 32) {
                            const int i = q0 + lane;
                            pkey_t k = 0;
                            unsigned sl2 = 0;
                            float tw2 = 0.f;
                            bool keep = false;
                            if (i < fn) {
                                const FEnt f = fe[i];
                                k = f.k;
                                sl2 = f.sl;
                                tw2 = f.tw;
                                const unsigned cur = hv[sl2];
                                keep = cur == dist_word((unsigned)(k >> 32));
                            }
                            const unsigned kb = __ballot_sync(0xffffffffu, keep);
                            __syncwarp();
                            if (keep) {
                                fe[w2 + __popc(kb & lt_mask)] = FEnt{k, sl2, tw2};
                            }
                            w2 += __popc(kb);
                            __syncwarp();
                        }
                        fn = w2;
                        if (fn + np > FS) overflow = true;
                    }
                    if (push && !overflow) {
                        const int p = fn + __popc(bal & lt_mask);
                        const pkey_t nk = make_key(nd, u);
                        const float tw = __fadd_rn(nd, __uint_as_float(uw));
                        fe[p] = FEnt{nk, slot, tw};
                        rk = nk < rk ? nk : rk;
                        rb = fminf(rb, tw);
                    }
                    fn += np;
                    overflow = __any_sync(0xffffffffu, overflow);
                    __syncwarp();
                    if (overflow) break;
                }
            }
            if (overflow) break;
        }
        if (overflow) {
            if (!RETRY) {
                // queued for the pass with large tables
                if (lane == 0) {
                    const unsigned q = atomicAdd(&st->knn_overflow, 1u);
                    if (q < (unsigned)a.total_matches)
                        a.knn_retry_list[q] = gm;
                    else
                        set_status(st, EPIC_ERR_CAPACITY);
                }
                __syncwarp();
                continue;
            }
            if (lane == 0) set_status(st, EPIC_ERR_CAPACITY);
            cnt = 0;
        }
        if (cnt > K) cnt = K;
        __syncwarp();
        // batches are appended in frontier order, which follows the order
        // of the adjacency rows (filled with atomics); sorting each batch by
        // key restores Dijkstra's settle order, so the fit below sums in a
        // canonical order and the result is bit-for-bit reproducible
        sort_settled(rn, rd, bs, cnt, reinterpret_cast<pkey_t *>(fe), lane);

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
            // Nadaraya-Watson sums (kernel k, not squared): k and k u_n
            acc_add(s[12], k);
            acc_prod(s[13], k, uh); s[13].lo = __fmaf_rn(k, ul, s[13].lo);
            acc_prod(s[14], k, vh); s[14].lo = __fmaf_rn(k, vl, s[14].lo);
        }
        // The totals are on every lane.  The float64 part runs lane-parallel:
        // float64 throughput is a small fraction of float32's here, and every
        // warp instruction costs the same however few lanes are active, so
        // each conversion, cofactor, quotient and coefficient goes to its own
        // lane and the operands travel by shuffles.
        // Transposed warp reduction of the 15 sums (a 16th is zero): at each
        // of four levels a lane keeps half of its items, sends the other half
        // to its partner and adds what it receives, so lanes 2i and 2i + 1
        // end with the partial sums of item i over 16 lanes each; one last
        // exchange completes them.  About 40 exchanges instead of 150.
        F2 mine;
        {
            F2 r[16];
#pragma unroll
            for (int i = 0; i < 15; ++i) r[i] = s[i];
            r[15] = F2{0.f, 0.f};
#pragma unroll
            for (int lvl = 0; lvl < 4; ++lvl) {
                const int m = 16 >> lvl, half = 8 >> lvl;
                const bool up = (lane & m) != 0;
#pragma unroll
                for (int j = 0; j < half; ++j) {
                    const F2 keep = up ? r[j + half] : r[j];
                    const F2 send = up ? r[j] : r[j + half];
                    const float oh = __shfl_xor_sync(0xffffffffu, send.hi, m);
                    const float ol = __shfl_xor_sync(0xffffffffu, send.lo, m);
                    float sh, eh;
                    two_sum(keep.hi, oh, sh, eh);
                    r[j] = F2{sh, __fadd_rn(keep.lo, __fadd_rn(ol, eh))};
                }
            }
            const float oh = __shfl_xor_sync(0xffffffffu, r[0].hi, 1);
            const float ol = __shfl_xor_sync(0xffffffffu, r[0].lo, 1);
            float sh, eh;
            two_sum(r[0].hi, oh, sh, eh);
            mine = F2{sh, __fadd_rn(r[0].lo, __fadd_rn(ol, eh))};
        }
        // lanes 2i and 2i + 1 hold sum i: M00 M01 M02 M11 M12 M22 (0-5), the
        // right-hand sides ru (6-8), rv (9-11), and the NW sums (12-14)
        const double Sl = to_d(mine);
        auto S = [&](int i) { return __shfl_sync(0xffffffffu, Sl, 2 * i); };
        // cofactors of the symmetric matrix M, c00 c01 c02 c11 c12 c22 on
        // lanes 0-5, each c = x y - z w with the operands' sum indices packed
        // in nibbles
        const int cj = lane < 6 ? lane : 0;
        const double cx = S((0x010143 >> (4 * cj)) & 15), cy = S((0x325425 >> (4 * cj)) & 15);
        const double cz = S((0x102314 >> (4 * cj)) & 15), cw = S((0x142254 >> (4 * cj)) & 15);
        const double Cl = __fma_rn(cx, cy, -__dmul_rn(cz, cw));
        auto Cf = [&](int src) { return __shfl_sync(0xffffffffu, Cl, src); };
        const double M00 = S(0), M01 = S(1), M02 = S(2), M11 = S(3), M22 = S(5);
        const double c00 = Cf(0), c01 = Cf(1), c02 = Cf(2);
        const double det = __fma_rn(M02, c02, __fma_rn(M01, c01, __dmul_rn(M00, c00)));
        const double tr = __dadd_rn(__dadd_rn(M00, M11), M22);
        // one division for four quotients: 1/det, the NW flow sum13/sum12
        // and sum14/sum12 (Eq. 1), and tr M / 3
        const double sk = S(12), s13 = S(13), s14 = S(14);
        const double qn = lane == 1 ? s13 : lane == 2 ? s14 : lane == 3 ? tr : 1.0;
        const double qd = lane == 0 ? det : lane == 3 ? 3.0 : lane < 3 ? sk : 1.0;
        const double q = qn / qd;
        const double id = __shfl_sync(0xffffffffu, q, 0);
        const double nwu = __shfl_sync(0xffffffffu, q, 1);
        const double nwv = __shfl_sync(0xffffffffu, q, 2);
        const double tr3 = __shfl_sync(0xffffffffu, q, 3);
        const bool fit_ok = a.estimator == 0 && cnt >= 3 &&
                            det > (double)a.fallback_eps * tr3 * tr3 * tr3;
        // affine coefficients bu0 bu1 bu2 bv0 bv1 bv2 on lanes 0-5:
        // (row k of the adjugate) . (ru or rv), times 1/det
        const int bk = lane < 6 ? lane : 0;
        const int rr = bk % 3, rbase = bk < 3 ? 6 : 9;
        const double bx0 = Cf(rr), bx1 = Cf(rr == 0 ? 1 : rr == 1 ? 3 : 4),
                     bx2 = Cf(rr == 0 ? 2 : rr == 1 ? 4 : 5);
        const double by0 = S(rbase), by1 = S(rbase + 1), by2 = S(rbase + 2);
        const float bl =
            (float)__dmul_rn(__fma_rn(bx2, by2, __fma_rn(bx1, by1, __dmul_rn(bx0, by0))), id);
        auto B = [&](int src) { return __shfl_sync(0xffffffffu, bl, src); };
        const float bu0 = B(0), bu1 = B(1), bu2 = B(2), bv0 = B(3), bv1 = B(4), bv2 = B(5);
        if (lane == 0) {
            float4 r0, r1;
            int fb;
            if (a.write_keep) {
                // consistency check (Sec. 4.1): keep the match when its own
                // flow is within the threshold of the NW estimate
                const double du = nwu - ((double)pm.z - (double)pm.x);
                const double dv = nwv - ((double)pm.w - (double)pm.y);
                const double thr = (double)a.prune_threshold;
                P.keep[m] = du * du + dv * dv <= thr * thr ? 1 : 0;
            }
            if (fit_ok) {
                r0 = make_float4(bu2, bv2, bu0, bu1);
                r1 = make_float4(bv0, bv1, pm.x, pm.y);
                fb = 0;
            } else {
                // the NW estimator, or the LA fit's fallback: the flow is
                // constant over the cell (Algorithm 1, step 8)
                r0 = make_float4((float)nwu, (float)nwv, 0.f, 0.f);
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

}  // namespace

// Main-pass tables: ~4.48 K node slots (the searches here touch about 1.5 K
// nodes; a sparse table keeps the probe sequences short) and ~1.6 K frontier
// entries (the largest frontier seen on these graphs is ~1.2 K), so that 8
// warps' tables fit four CTAs on an SM up to K ~ 100.  For larger K the
// tables shrink to what four CTAs leave: 7/8 of an equal split to the
// frontier (at least 1.4 K entries), the rest to the node table; beyond
// that (K above ~160) they keep the proportions ~3.84 K and ~1.92 K at fewer
// CTAs per SM.  A search that outgrows them is run again with large tables.
void knn_table_sizes(int max_K, const LaunchCfg &lc, int *hs, int *fs) {
    const int k = max_K > 1 ? max_K : 1;
    *hs = std::max(64, (k * 448 / 100 + 31) / 32 * 32);
    *fs = std::max(64, (k * 160 / 100 + 31) / 32 * 32);
    if (lc.smem_per_sm <= 0) return;
    const long long per_warp = ((long long)lc.smem_per_sm / 4 - lc.smem_reserved) / KNN_WARPS;
    const long long fixed = (long long)knn_fixed_bytes(k);
    if ((long long)*fs * 16 + (long long)*hs * 8 + fixed <= per_warp) return;
    const long long f = (per_warp - fixed) / 32;   // 16 B per entry + 2 slots of 8 B
    if (f * 10 >= 14LL * k) {
        *fs = (int)(f * 7 / 8);
        *hs = (int)((per_warp - fixed - (long long)*fs * 16) / 8);
        return;
    }
    // fewer CTAs per SM: tables in proportion to K (~3.84 K slots, ~1.92 K
    // entries), which stay below the retry pass's up to EPIC_MAX_K
    *hs = std::max(64, (k * 384 / 100 + 31) / 32 * 32);
    *fs = std::max(64, (k * 192 / 100 + 31) / 32 * 32);
}

// Retry-pass tables: the largest power-of-two node table (and a frontier
// half its size) whose tables fit one warp per CTA.
void knn_retry_table_sizes(int max_K, int smem_limit, int *hs, int *fs) {
    int h = 64;
    while (knn_warp_bytes(2 * h, h, max_K) <= (size_t)smem_limit && h < (1 << 20)) h *= 2;
    *hs = h;
    *fs = h / 2;
}

size_t knn_smem_per_warp(int max_K, const LaunchCfg &lc) {
    int hs, fs;
    knn_table_sizes(max_K, lc, &hs, &fs);
    return knn_warp_bytes(hs, fs, max_K);
}

// Largest warps-per-CTA (<= KNN_WARPS) whose tables fit in shared memory;
// 0 if even one warp's tables do not fit.
int knn_warps_per_cta(int max_K, const LaunchCfg &lc) {
    size_t pw = knn_smem_per_warp(max_K, lc);
    int w = (int)(lc.smem_optin / pw);
    return w > KNN_WARPS ? KNN_WARPS : w;
}

cudaError_t launch_knn_fit(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc,
                           int max_K) {
    (void)a;
    int warps = knn_warps_per_cta(max_K, lc);
    if (warps < 1) return cudaErrorInvalidValue;
    int hs, fs, rhs, rfs;
    knn_table_sizes(max_K, lc, &hs, &fs);
    knn_retry_table_sizes(max_K, lc.smem_optin, &rhs, &rfs);
    const size_t smem = knn_warp_bytes(hs, fs, max_K) * warps;
    const size_t rsmem = knn_warp_bytes(rhs, rfs, max_K);
    cudaError_t e = cudaFuncSetAttribute(knn_fit_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(knn_fit_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rsmem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, knn_fit_kernel<false>,
                                                      warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    knn_fit_kernel<false><<<per_sm * lc.num_sms, warps * 32, smem, lc.stream>>>(dev, hs, fs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the queued matches (usually none: every CTA returns at once)
    knn_fit_kernel<true><<<lc.num_sms, 32, rsmem, lc.stream>>>(dev, rhs, rfs);
    return cudaGetLastError();
}

}  // namespace epic
