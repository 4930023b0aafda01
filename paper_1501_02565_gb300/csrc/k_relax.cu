// Stage (a) of the interpolator: geodesic assignment map L and distance D
// (Sec. 3.4 "Geodesic Voronoi diagram"; D_G of Eq. 3 on the 8-connected
// grid) by row-closure passes on warp-owned tiles.
//
// The keys are the same exact fixed-point (D, L) keys as in k_dt.cu, so any
// order of relaxation steps that ends when no step improves any key reaches
// the same keys bit for bit; this kernel reaches them with far fewer steps.
//
// Tiles are 64 columns x R rows (R <= 32, one frame's rows per tile from its
// tile rule); each warp is an independent worker that takes whole tiles from
// a counter and solves them in its own shared memory, lane l holding columns
// 2l and 2l+1.  A tile solve alternates two kinds of pass:
//
//   down  rows top to bottom: row y takes the three candidates from the row
//         above (already final in this pass), then is closed along itself --
//         every pixel takes the best of its row neighbours' keys plus the
//         exact axis steps, repeated until nothing changes -- so that after
//         the pass every pixel holds its best key over all paths that never
//         move up;
//   up    the same from the bottom row upwards.
//
// Per-row flags record which constraints may be violated: a row must be
// stepped in a down pass only if the row above changed since it was last
// stepped downwards, or if its own ring neighbours or seeds demand it (and
// likewise upwards).  A tile is solved when every flag is clear; no pass is
// run only to confirm.
//
// One launch holds the whole relaxation (a cooperative launch, every CTA
// resident):
//   phase 1  every tile is solved from its own seeds, in two halves of a
//            chessboard: first the tiles with tx + ty even, with unreached
//            neighbours around them, then the others, with the first half's
//            results in their ring (so their solves start from distances
//            that already cross the tile borders, and fewer re-solves
//            follow);
//   phase 2  a work queue of tiles: every tile once (the sweep), then every
//            tile asked for by a neighbour whose border keys changed.  A
//            solve loads the tile and the ring of pixels around it, sets the
//            flags of the rows its ring can improve and re-solves if any.
//            The phase ends when nothing is queued or being solved, i.e. no
//            step improves any key anywhere; no grid barrier divides it, so
//            a front of changes moves on through the tiles as soon as each
//            one is solved.
// Nor does a grid barrier divide the phases or the halves: a second-half
// tile waits for its four edge neighbours' stamps, and a phase-2 solve for
// the stamps of the tile and its eight neighbours (every wait bounded; the
// prepare kernel marks the tiles pending at the start of a run).
#include "epic_internal.cuh"

namespace epic {

namespace {

constexpr int RT_COLS = 64;   // tile width: two columns per lane
constexpr int RT_WARPS = 1;   // warps (tile workers) per CTA
constexpr unsigned FULL = 0xFFFFFFFFu;
// shared-memory row pitches, as the TMA boxes land them: keys from column
// x0 - 2 (68 x 8 bytes; the tile at 2..65, ring columns at 1 and 66) and
// costs from column x0 - 4 (72 x 4 bytes; the tile at 4..67, ring columns at
// 3 and 68), so a lane's two keys are one aligned 16-byte access
constexpr int KP = 68, KO = 2;
constexpr int CP = 72, CO = 4;
constexpr unsigned long long TMA_LIMIT_NS = 1000000000ull;  // 1 s
constexpr int SCAN_CHUNK = 4;   // most tiles a warp takes at once in the passes of phase 2

// One warp's tile in shared memory.  Row r is image row y0 - 1 + r, so rows
// 0 and R + 1 are the ring rows above and below.  hC holds the costs as
// staged, then the half-costs (as unsigned bits) after conversion.
template <int MAXR>
struct WarpTile {
    alignas(128) pkey_t K[MAXR + 2][KP];       // TMA destinations are 128-byte aligned
    alignas(128) unsigned hC[MAXR + 2][CP];
    unsigned long long bar;   // mbarrier of the warp's TMA copies
};
static_assert(sizeof(WarpTile<8>) % 128 == 0 && sizeof(WarpTile<16>) % 128 == 0 &&
                  sizeof(WarpTile<32>) % 128 == 0,
              "warp tiles stay 128-byte aligned in an array");

__device__ __forceinline__ pkey_t kmin(pkey_t a, pkey_t b) { return b < a ? b : a; }

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long x) {
    const unsigned lo = __reduce_or_sync(FULL, (unsigned)x);
    const unsigned hi = __reduce_or_sync(FULL, (unsigned)(x >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

// Tile geometry of one solve.
struct TileGeo {
    int x0, y0;     // image origin
    int wv, rv;     // valid columns (<= 64) and rows (<= R)
    bool outa, outb;  // this lane's columns lie outside the image
};

__device__ __forceinline__ TileGeo tile_geo(const PairDev &P, int tx, int ty, int lane) {
    TileGeo g;
    g.x0 = tx * RT_COLS;
    g.y0 = ty * P.tile_h;
    g.wv = min(RT_COLS, P.W - g.x0);
    g.rv = min(P.tile_h, P.H - g.y0);
    g.outa = 2 * lane >= g.wv;
    g.outb = 2 * lane + 1 >= g.wv;
    return g;
}

// The upstream row yu as seen by this lane: its two keys and half-costs and
// those of the columns on either side (a neighbour lane's, or the ring).
struct Up {
    pkey_t Pa, Pb, lK, rK;
    unsigned pha, phb, lh, rh;
};

template <int MAXR>
__device__ __forceinline__ void load_up(const WarpTile<MAXR> &T, int yu, int lane, Up &u) {
    const ulonglong2 kk = *reinterpret_cast<const ulonglong2 *>(&T.K[yu][KO + 2 * lane]);
    const uint2 hh = *reinterpret_cast<const uint2 *>(&T.hC[yu][CO + 2 * lane]);
    u.Pa = kk.x;
    u.Pb = kk.y;
    u.pha = hh.x;
    u.phb = hh.y;
}

template <int MAXR>
__device__ __forceinline__ void neighbours_up(const WarpTile<MAXR> &T, int yu, int lane, Up &u) {
    const pkey_t l = __shfl_up_sync(FULL, u.Pb, 1);
    const unsigned lh = __shfl_up_sync(FULL, u.phb, 1);
    const pkey_t r = __shfl_down_sync(FULL, u.Pa, 1);
    const unsigned rh = __shfl_down_sync(FULL, u.pha, 1);
    u.lK = lane == 0 ? T.K[yu][KO - 1] : l;
    u.lh = lane == 0 ? T.hC[yu][CO - 1] : lh;
    u.rK = lane == 31 ? T.K[yu][KO + RT_COLS] : r;
    u.rh = lane == 31 ? T.hC[yu][CO + RT_COLS] : rh;
}

// Best keys of this lane's two pixels of a row (keys Ka, Kb, half-costs ha,
// hb) over their current keys and the three candidates each from row u.
__device__ __forceinline__ void from_up(const Up &u, pkey_t Ka, pkey_t Kb, unsigned ha,
                                        unsigned hb, pkey_t &na, pkey_t &nb) {
    na = kmin(Ka, step_key(u.Pa, step_axis(ha, u.pha)));
    na = kmin(na, step_key(u.lK, step_diag(ha, u.lh)));
    na = kmin(na, step_key(u.Pb, step_diag(ha, u.phb)));
    nb = kmin(Kb, step_key(u.Pb, step_axis(hb, u.phb)));
    nb = kmin(nb, step_key(u.Pa, step_diag(hb, u.pha)));
    nb = kmin(nb, step_key(u.rK, step_diag(hb, u.rh)));
}

// A row as one step of a stream reads it: this lane's two keys and
// half-costs, the half-costs of the columns on either side and the ring keys.
struct RowIn {
    ulonglong2 kk;
    unsigned ha, hb, hl, hr;
    pkey_t ringl, ringr;
};

template <int MAXR>
__device__ __forceinline__ void row_in(const WarpTile<MAXR> &T, int y, int lane, RowIn &r) {
    r.kk = *reinterpret_cast<const ulonglong2 *>(&T.K[y][KO + 2 * lane]);
    const uint2 hh = *reinterpret_cast<const uint2 *>(&T.hC[y][CO + 2 * lane]);
    r.ha = hh.x;
    r.hb = hh.y;
    r.ringl = T.K[y][KO - 1];
    r.ringr = T.K[y][KO + RT_COLS];
    const unsigned hl0 = __shfl_up_sync(FULL, r.hb, 1);
    const unsigned hr0 = __shfl_down_sync(FULL, r.ha, 1);
    r.hl = lane == 0 ? T.hC[y][CO - 1] : hl0;
    r.hr = lane == 31 ? T.hC[y][CO + RT_COLS] : hr0;
}

// The row's own step weights: left neighbour to a, a to b, b to right.
struct RowW {
    unsigned long long wl, wab, wr;
};

__device__ __forceinline__ RowW row_w(const RowIn &r) {
    return RowW{step_axis(r.hl, r.ha), step_axis(r.ha, r.hb), step_axis(r.hb, r.hr)};
}

// One closure round along a row: each lane sweeps its pair left to right and
// back with its neighbours' keys of the previous round (the ring columns
// fixed).  Returns whether this lane's keys changed.
__device__ __forceinline__ bool close_round(pkey_t &na, pkey_t &nb, const RowIn &r,
                                            const RowW &w, int lane, const TileGeo &g) {
    pkey_t left = __shfl_up_sync(FULL, nb, 1);
    pkey_t right = __shfl_down_sync(FULL, na, 1);
    if (lane == 0) left = r.ringl;
    if (lane == 31) right = r.ringr;
    pkey_t a2 = kmin(na, step_key(left, w.wl));
    pkey_t b2 = kmin(nb, step_key(a2, w.wab));
    b2 = kmin(b2, step_key(right, w.wr));
    a2 = kmin(a2, step_key(b2, w.wab));
    if (g.outa) a2 = KEY_INF;
    if (g.outb) b2 = KEY_INF;
    const bool ch = (a2 != na) | (b2 != nb);
    na = a2;
    nb = b2;
    return ch;
}

// The vertical part of a step: this lane's two pixels take the three
// candidates each from the upstream row u.  Returns whether the row must be
// closed along itself: it is stepped for its own sake (must_close: seeds,
// ring neighbours; it may not be closed yet), or the upstream row improved
// one of its pixels (otherwise it is unchanged, and it was closed when it
// was last stepped).
__device__ __forceinline__ bool row_from_up(const Up &u, const RowIn &r, const TileGeo &g,
                                            bool must_close, pkey_t &na, pkey_t &nb) {
    from_up(u, r.kk.x, r.kk.y, r.ha, r.hb, na, nb);
    if (g.outa) na = KEY_INF;
    if (g.outb) nb = KEY_INF;
    return must_close || __any_sync(FULL, (na != r.kk.x) | (nb != r.kk.y));
}

// Closure rounds until a round changes nothing anywhere (at most one round
// per two columns, plus one).
__device__ __forceinline__ void close_row(pkey_t &na, pkey_t &nb, const RowIn &r, int lane,
                                          const TileGeo &g) {
    const RowW w = row_w(r);
    for (int round = 0; round <= RT_COLS / 2 + 1; ++round)
        if (!__any_sync(FULL, close_round(na, nb, r, w, lane, g))) break;
}

// Ends a step of row y: writes the row back if it changed and leaves it in
// u (the upstream row of the stream's next step).  Returns whether it changed.
template <int MAXR>
__device__ __forceinline__ bool row_out(WarpTile<MAXR> &T, int y, int lane, const RowIn &r,
                                        pkey_t na, pkey_t nb, Up &u, unsigned &edges) {
    const bool changed = __any_sync(FULL, (na != r.kk.x) | (nb != r.kk.y));
    if (changed) {
        *reinterpret_cast<ulonglong2 *>(&T.K[y][KO + 2 * lane]) = make_ulonglong2(na, nb);
        // bit 0: column 0 changed; bit 1: column 63
        edges |= (__ballot_sync(FULL, na != r.kk.x) & 1u) |
                 ((__ballot_sync(FULL, nb != r.kk.y) >> 30) & 2u);
    }
    u.Pa = na;
    u.Pb = nb;
    u.pha = r.ha;
    u.phb = r.hb;
    return changed;
}

// Step row y from the upstream row (registers u, with neighbours): three
// candidates per pixel, then the closure along the row.  Returns whether the
// row changed; on return u holds row y.
template <int MAXR>
__device__ __forceinline__ bool row_step(WarpTile<MAXR> &T, int y, int lane, const TileGeo &g,
                                         Up &u, bool must_close, unsigned &edges) {
    RowIn r;
    row_in(T, y, lane, r);
    pkey_t na, nb;
    if (row_from_up(u, r, g, must_close, na, nb)) close_row(na, nb, r, lane, g);
    return row_out(T, y, lane, r, na, nb, u, edges);
}

// Down and up passes over rows 1..rv until every flag is clear.  forD bit r:
// row r changed since row r + 1 was last stepped downwards (forU: upwards,
// row r - 1); selfD / selfU bit r: row r must be stepped in the next down /
// up pass for its own sake (seeds, ring neighbours).  Returns the mask of
// rows that changed; `edges` gains bit 0 (1) if column 0 (63) changed.
template <int MAXR>
__device__ unsigned long long tile_passes(WarpTile<MAXR> &T, int lane, const TileGeo &g,
                                          unsigned long long forD, unsigned long long forU,
                                          unsigned long long selfD, unsigned long long selfU,
                                          RunState *st, unsigned &edges) {
    const int rv = g.rv;
    const unsigned long long ring = 1ull | (1ull << (rv + 1));
    unsigned long long modified = 0;
    // each pass that changes a row undoes one turn of some shortest path, and
    // a path in the tile has fewer turns than pixels
    const int cap = 2 + RT_COLS * rv;
    for (int pass = 0;; ++pass) {
        // a ring row is never stepped, so what it would consume is dropped
        forD &= ~((1ull << rv) | ring);
        forU &= ~(2ull | ring);
        if ((forD | forU | selfD | selfU) == 0) break;
        if (pass >= cap) {
            if (lane == 0) set_status(st, EPIC_ERR_NOT_CONVERGED);
            break;
        }
        const bool down = (pass & 1) == 0;
        Up u;
        int have = -1;   // row whose values u holds
        for (int i = 1; i <= rv; ++i) {
            const int y = down ? i : rv + 1 - i;
            const int yu = down ? y - 1 : y + 1;
            unsigned long long &fl = down ? forD : forU;
            unsigned long long &sf = down ? selfD : selfU;
            const bool self = (sf >> y) & 1ull;
            if (!(((fl >> yu) & 1ull) | self)) continue;
            fl &= ~(1ull << yu);
            sf &= ~(1ull << y);
            if (have != yu) load_up(T, yu, lane, u);
            neighbours_up(T, yu, lane, u);
            if (row_step(T, y, lane, g, u, self, edges)) {
                forD |= 1ull << y;
                forU |= 1ull << y;
                modified |= 1ull << y;
            }
            have = y;
        }
    }
    return modified;
}

// Can this lane read (write) its two cells of image row gy with one vector
// access?  The keys (arena, 256-byte aligned) need an even offset; the
// caller's cost map also an 8-byte-aligned base.
__device__ __forceinline__ bool row_vec_ok(int gy, int W) { return ((gy * (long long)W) & 1) == 0; }
__device__ __forceinline__ bool cost_vec_ok(const PairDev &P, int gy) {
    return row_vec_ok(gy, P.W) && ((uintptr_t)P.C & 7) == 0;
}

// Write rows `rows` (bit r = tile row r) of the tile back to the key map.
template <int MAXR>
__device__ void write_rows(const PairDev &P, const WarpTile<MAXR> &T, const TileGeo &g,
                           unsigned long long rows, int lane) {
    const int c = 2 * lane;
    while (rows) {
        const int r = __ffsll((long long)rows) - 1;
        rows &= rows - 1;
        const int gy = g.y0 + r - 1;
        pkey_t *dst = P.keys + (size_t)gy * P.W + g.x0 + c;
        const ulonglong2 kk = *reinterpret_cast<const ulonglong2 *>(&T.K[r][KO + c]);
        if (c + 1 < g.wv && row_vec_ok(gy, P.W)) {
            *reinterpret_cast<ulonglong2 *>(dst) = kk;
        } else {
            if (c < g.wv) dst[0] = kk.x;
            if (c + 1 < g.wv) dst[1] = kk.y;
        }
    }
}

__device__ __forceinline__ unsigned long long warp_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// TMA staging of one tile: lane 0 starts the box copies of the keys (if
// `keys`) and the costs into the warp's tile, completing on its mbarrier;
// every lane then waits, at most TMA_LIMIT_NS.  Returns false in every lane
// if the wait gave up (the run has recorded EPIC_ERR_TIMEOUT; a copy may
// still land in this CTA's shared memory after the kernel has left).
template <int MAXR>
__device__ bool tma_stage(const PairDev &P, WarpTile<MAXR> &T, const TileGeo &g, bool keys,
                          unsigned &phase, int lane, RunState *st) {
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&T.bar);
    __syncwarp();   // every lane is done with the previous tile's data
    if (lane == 0) {
        const unsigned kbytes = (unsigned)(KP * (P.tile_h + 2) * 8);
        const unsigned cbytes = (unsigned)(CP * (P.tile_h + 2) * 4);
        // the keys were written by other CTAs with generic stores (ordered
        // before this point by the stamps and the grid barrier); the bulk
        // copies read them through the async proxy
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(cbytes + (keys ? kbytes : 0u))
                     : "memory");
        const int y = g.y0 - 1;
        if (keys) {
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                             &P.tm_warp_keys)
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3}], [%4];" ::"r"((unsigned)__cvta_generic_to_shared(&T.K[0][0])),
                "l"(&P.tm_warp_keys), "r"(g.x0 - KO), "r"(y), "r"(bar)
                : "memory");
        }
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&P.tm_warp_cost)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];" ::"r"((unsigned)__cvta_generic_to_shared(&T.hC[0][0])),
            "l"(&P.tm_warp_cost), "r"(g.x0 - CO), "r"(y), "r"(bar)
            : "memory");
    }
    const unsigned long long t0 = warp_ns();
    int gave_up = 0;
    for (;;) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
            " selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) break;
        if (warp_ns() - t0 > TMA_LIMIT_NS) {
            set_status(st, EPIC_ERR_TIMEOUT);
            gave_up = 1;
            break;
        }
    }
    phase ^= 1u;
    return !__any_sync(FULL, gave_up);
}

// Plain-load staging into the same layout (maps whose pitch or base does
// not meet TMA's 16-byte rules).  Keys and costs outside the image read as
// unreached and zero.  Keys of other tiles may be rewritten during the
// launch: they are read through L2.
template <int MAXR>
__device__ void plain_stage(const PairDev &P, WarpTile<MAXR> &T, const TileGeo &g, bool keys,
                            int lane) {
    const int c = 2 * lane;
    for (int r = 0; r <= g.rv + 1; ++r) {
        const int gy = g.y0 + r - 1;
        ulonglong2 kk = make_ulonglong2(KEY_INF, KEY_INF);
        uint2 cc = make_uint2(0u, 0u);
        if (gy >= 0 && gy < P.H) {
            const size_t o = (size_t)gy * P.W + g.x0 + c;
            if (c + 1 < g.wv && cost_vec_ok(P, gy)) {
                if (keys) kk = __ldcg(reinterpret_cast<const ulonglong2 *>(P.keys + o));
                const float2 f = __ldg(reinterpret_cast<const float2 *>(P.C + o));
                cc = make_uint2(__float_as_uint(f.x), __float_as_uint(f.y));
            } else {
                if (c < g.wv) {
                    if (keys) kk.x = __ldcg(P.keys + o);
                    cc.x = __float_as_uint(__ldg(P.C + o));
                }
                if (c + 1 < g.wv) {
                    if (keys) kk.y = __ldcg(P.keys + o + 1);
                    cc.y = __float_as_uint(__ldg(P.C + o + 1));
                }
            }
        }
        if (keys) *reinterpret_cast<ulonglong2 *>(&T.K[r][KO + c]) = kk;
        *reinterpret_cast<uint2 *>(&T.hC[r][CO + c]) = cc;
    }
    for (int r = lane; r < g.rv + 2; r += 32) {
        const int gy = g.y0 + r - 1;
        const bool row_in = gy >= 0 && gy < P.H;
        pkey_t kl = KEY_INF, kr = KEY_INF;
        unsigned cl = 0u, cr = 0u;
        if (row_in && g.x0 > 0) {
            const size_t o = (size_t)gy * P.W + g.x0 - 1;
            if (keys) kl = __ldcg(P.keys + o);
            cl = __float_as_uint(__ldg(P.C + o));
        }
        if (row_in && g.x0 + RT_COLS < P.W) {
            const size_t o = (size_t)gy * P.W + g.x0 + RT_COLS;
            if (keys) kr = __ldcg(P.keys + o);
            cr = __float_as_uint(__ldg(P.C + o));
        }
        if (keys) {
            T.K[r][KO - 1] = kl;
            T.K[r][KO + RT_COLS] = kr;
        }
        T.hC[r][CO - 1] = cl;
        T.hC[r][CO + RT_COLS] = cr;
    }
}

// Stage tile (tx, ty) and its ring: keys (if `keys`, else unreached) and
// half-costs.  Cells outside the image end as unreached keys and zero
// half-costs, whichever way they were copied.  Returns false when a TMA
// wait gave up (the caller leaves the kernel).
template <int MAXR>
__device__ bool stage_tile(const PairDev &P, WarpTile<MAXR> &T, const TileGeo &g, bool keys,
                           unsigned &phase, int lane, RunState *st) {
    const int c = 2 * lane;
    if (P.tma_warp) {
        if (!tma_stage(P, T, g, keys, phase, lane, st)) return false;
    } else {
        __syncwarp();
        plain_stage(P, T, g, keys, lane);
    }
    bool bad = false;
    const int us = unit_shift(P);   // the pair's distance unit
    for (int r = 0; r <= g.rv + 1; ++r) {
        const int gy = g.y0 + r - 1;
        const bool row_in = gy >= 0 && gy < P.H;
        // keys: a fresh tile starts unreached; out-of-image cells are
        // unreached (TMA fills them with zeros)
        ulonglong2 kk = *reinterpret_cast<const ulonglong2 *>(&T.K[r][KO + c]);
        if (!keys || !row_in || g.outa) kk.x = KEY_INF;
        if (!keys || !row_in || g.outb) kk.y = KEY_INF;
        *reinterpret_cast<ulonglong2 *>(&T.K[r][KO + c]) = kk;
        // half-costs, in place
        uint2 cc = *reinterpret_cast<const uint2 *>(&T.hC[r][CO + c]);
        cc.x = row_in && !g.outa ? half_cost_s(__uint_as_float(cc.x), us, &bad) : 0u;
        cc.y = row_in && !g.outb ? half_cost_s(__uint_as_float(cc.y), us, &bad) : 0u;
        *reinterpret_cast<uint2 *>(&T.hC[r][CO + c]) = cc;
    }
    for (int r = lane; r < g.rv + 2; r += 32) {
        const int gy = g.y0 + r - 1;
        const bool row_in = gy >= 0 && gy < P.H;
        const bool lin = row_in && g.x0 > 0, rin = row_in && g.x0 + RT_COLS < P.W;
        if (!keys || !lin) T.K[r][KO - 1] = KEY_INF;
        if (!keys || !rin) T.K[r][KO + RT_COLS] = KEY_INF;
        T.hC[r][CO - 1] = lin ? half_cost_s(__uint_as_float(T.hC[r][CO - 1]), us, &bad) : 0u;
        T.hC[r][CO + RT_COLS] = rin ? half_cost_s(__uint_as_float(T.hC[r][CO + RT_COLS]), us, &bad) : 0u;
    }
    if (__any_sync(FULL, bad) && lane == 0) set_status(st, EPIC_ERR_INVALID);
    __syncwarp();
    return true;
}

// Rows of the staged tile that a ring pixel can improve by one step: the top
// row from ring row 0 (a down step of row 1), the bottom row from ring row
// rv + 1 (an up step of row rv); the end columns of row r from the ring
// column in rows r - 1 and r (a down step) and r + 1 (an up step).
template <int MAXR>
__device__ void ring_flags(const WarpTile<MAXR> &T, const TileGeo &g, int lane,
                           unsigned long long &selfD, unsigned long long &selfU) {
    const int c = 2 * lane;
    {
        Up u;
        pkey_t na, nb;
        load_up(T, 0, lane, u);
        neighbours_up(T, 0, lane, u);
        const ulonglong2 k1 = *reinterpret_cast<const ulonglong2 *>(&T.K[1][KO + c]);
        const uint2 h1 = *reinterpret_cast<const uint2 *>(&T.hC[1][CO + c]);
        from_up(u, k1.x, k1.y, h1.x, h1.y, na, nb);
        const bool top = (!g.outa && na < k1.x) || (!g.outb && nb < k1.y);
        load_up(T, g.rv + 1, lane, u);
        neighbours_up(T, g.rv + 1, lane, u);
        const ulonglong2 kb = *reinterpret_cast<const ulonglong2 *>(&T.K[g.rv][KO + c]);
        const uint2 hb = *reinterpret_cast<const uint2 *>(&T.hC[g.rv][CO + c]);
        from_up(u, kb.x, kb.y, hb.x, hb.y, na, nb);
        const bool bot = (!g.outa && na < kb.x) || (!g.outb && nb < kb.y);
        if (__any_sync(FULL, top)) selfD |= 2ull;
        if (__any_sync(FULL, bot)) selfU |= 1ull << g.rv;
    }
    {
        // lane r - 1 looks at row r's end columns (rv <= 32 rows)
        const int r = lane + 1;
        bool d = false, up = false;
        if (r <= g.rv) {
            const pkey_t k0 = T.K[r][KO];
            const unsigned h0 = T.hC[r][CO];
            const int L = KO - 1, LC = CO - 1;
            d |= step_key(T.K[r - 1][L], step_diag(h0, T.hC[r - 1][LC])) < k0;
            d |= step_key(T.K[r][L], step_axis(h0, T.hC[r][LC])) < k0;
            up |= step_key(T.K[r + 1][L], step_diag(h0, T.hC[r + 1][LC])) < k0;
            if (g.wv == RT_COLS) {
                const pkey_t k1 = T.K[r][KO + RT_COLS - 1];
                const unsigned h1 = T.hC[r][CO + RT_COLS - 1];
                const int R = KO + RT_COLS, RC = CO + RT_COLS;
                d |= step_key(T.K[r - 1][R], step_diag(h1, T.hC[r - 1][RC])) < k1;
                d |= step_key(T.K[r][R], step_axis(h1, T.hC[r][RC])) < k1;
                up |= step_key(T.K[r + 1][R], step_diag(h1, T.hC[r + 1][RC])) < k1;
            }
        }
        selfD |= (unsigned long long)__ballot_sync(FULL, d) << 1;
        selfU |= (unsigned long long)__ballot_sync(FULL, up) << 1;
    }
}

// Phase 1: solve tile (tx, ty) from its own seeds.  The first half of the
// phase takes the tiles with tx + ty even, alone (an unreached ring); the
// second half the others (ring = true), which stage the ring from their
// four edge neighbours, solved by then (the corner pixels of the ring
// belong to tiles of the second half and stay unreached).  A tile with
// nothing to solve (no seeds, and for the second half no ring pixel that
// improves it) is written unreached and stamped "never written" (-1), so
// that in the first pass its seedless neighbours skip it.  Returns false
// when the staging timed out.
template <int MAXR>
__device__ bool fresh_tile(const PairDev &P, int t, int tx, int ty, WarpTile<MAXR> &T, int lane,
                           unsigned &phase, RunState *st, bool ring) {
    const TileGeo g = tile_geo(P, tx, ty, lane);
    const int c = 2 * lane;
    const int s0 = P.tile_start[t], s1 = P.tile_start[t + 1];
    const unsigned long long all = ((1ull << g.rv) - 1) << 1;
    if (s0 == s1 && !ring) {
        __syncwarp();
        for (int r = 1; r <= g.rv; ++r)
            *reinterpret_cast<ulonglong2 *>(&T.K[r][KO + c]) = make_ulonglong2(KEY_INF, KEY_INF);
        __syncwarp();
        write_rows(P, T, g, all, lane);
        __threadfence();
        if (lane == 0) P.tile_stamp[t] = -1;
        __syncwarp();
        return true;
    }
    if (!stage_tile(P, T, g, ring, phase, lane, st)) return false;
    unsigned long long selfD = 0, selfU = 0;
    if (ring) {
        // the tile itself starts unreached, and so do the ring's corners
        for (int r = 1; r <= g.rv; ++r)
            *reinterpret_cast<ulonglong2 *>(&T.K[r][KO + c]) = make_ulonglong2(KEY_INF, KEY_INF);
        if (lane < 4) T.K[lane < 2 ? 0 : g.rv + 1][lane & 1 ? KO + RT_COLS : KO - 1] = KEY_INF;
        __syncwarp();
        ring_flags(T, g, lane, selfD, selfU);
    }
    unsigned long long seeded = 0;
    for (int s = s0 + lane; s < s1; s += 32) {
        const int m = P.tile_seeds[s];
        const float4 mt = __ldg(P.matches + m);
        const int px = (int)floorf(mt.x + 0.5f) - g.x0;
        const int py = (int)floorf(mt.y + 0.5f) - g.y0;
        if (px >= 0 && px < g.wv && py >= 0 && py < g.rv) {
            atomicMin(&T.K[py + 1][KO + px],
                      make_key(P.seed_init ? P.seed_init[m] : 0ull, (unsigned)m));
            seeded |= 1ull << (py + 1);
        }
    }
    seeded = warp_or64(seeded);
    __syncwarp();
    if ((seeded | selfD | selfU) == 0) {
        // second half, no seeds, and the ring reaches nothing
        write_rows(P, T, g, all, lane);
        __threadfence();
        if (lane == 0) P.tile_stamp[t] = -1;
        __syncwarp();
        return true;
    }
    unsigned edges = 0;
    tile_passes(T, lane, g, seeded, seeded, seeded | selfD, selfU, st, edges);
    __syncwarp();
    write_rows(P, T, g, all, lane);
    __threadfence();
    if (lane == 0) P.tile_stamp[t] = 0;
    __syncwarp();
    return true;
}

// Phase 2: stage tile (tx, ty) with its ring from the current key map, set
// the flags of the rows the ring can improve and re-solve.  Returns 1 if any
// key of the tile changed (then it was written back and stamped `stamp`),
// 0 if none did, -1 if the staging timed out; *modified gets the mask of
// changed tile rows (bit r = row r), *edges bit 0 (1) whether column 0 (63)
// changed.
template <int MAXR>
__device__ int resolve_tile(const PairDev &P, int t, int tx, int ty, WarpTile<MAXR> &T,
                            int lane, unsigned &phase, RunState *st, int stamp,
                            unsigned long long *modified, unsigned *edges) {
    *modified = 0;
    *edges = 0;
    const TileGeo g = tile_geo(P, tx, ty, lane);
    if (!stage_tile(P, T, g, true, phase, lane, st)) return -1;
    unsigned long long selfD = 0, selfU = 0;
    ring_flags(T, g, lane, selfD, selfU);
    if ((selfD | selfU) == 0) return 0;
    const unsigned long long mod = tile_passes(T, lane, g, 0ull, 0ull, selfD, selfU, st, *edges);
    *modified = mod;
    if (mod == 0) return 0;
    __syncwarp();
    write_rows(P, T, g, mod, lane);
    __threadfence();
    if (lane == 0) P.tile_stamp[t] = stamp;
    __syncwarp();
    return 1;
}

// Waits until the four edge neighbours of tile (tx, ty) (those inside the
// tile grid) carry a stamp of this run, i.e. are written; lane k < 4 watches
// one.  Gives up after TMA_LIMIT_NS with EPIC_ERR_TIMEOUT (false in every
// lane).
__device__ bool wait_edge_neighbours(const PairDev &P, int tx, int ty, int lane, RunState *st) {
    bool gave_up = false;
    if (lane < 4) {
        const int x = tx + (lane == 0 ? -1 : lane == 1 ? 1 : 0);
        const int y = ty + (lane == 2 ? -1 : lane == 3 ? 1 : 0);
        if (x >= 0 && x < P.tiles_x && y >= 0 && y < P.tiles_y) {
            const unsigned *sp = reinterpret_cast<const unsigned *>(P.tile_stamp + y * P.tiles_x + x);
            const unsigned long long t0 = warp_ns();
            while (ld_acquire(sp) == (unsigned)STAMP_PENDING) {
                if (warp_ns() - t0 > TMA_LIMIT_NS) {
                    set_status(st, EPIC_ERR_TIMEOUT);
                    gave_up = true;
                    break;
                }
            }
        }
    }
    return !__any_sync(FULL, gave_up);
}

// Waits until tile (tx, ty) and its eight neighbours (those inside the tile
// grid) carry a stamp of this run (phase 1 has written them); lane k < 8
// watches neighbour k, lane 8 the tile.  Then, for the sweep (`any_written`
// not null), tells whether any neighbour was reached (stamp >= 0).  Gives up
// after TMA_LIMIT_NS with EPIC_ERR_TIMEOUT (false in every lane).
__device__ bool wait_tile_and_ring(const PairDev &P, int tx, int ty, int lane, RunState *st,
                                   bool *any_written) {
    bool gave_up = false, written = false;
    if (lane < 9) {
        const int x = lane == 8 ? tx : tx + (lane < 3 ? lane - 1 : lane < 5 ? 2 * lane - 7 : lane - 6);
        const int y = lane == 8 ? ty : ty + (lane < 3 ? -1 : lane < 5 ? 0 : 1);
        if (x >= 0 && x < P.tiles_x && y >= 0 && y < P.tiles_y) {
            const unsigned *sp = reinterpret_cast<const unsigned *>(P.tile_stamp + y * P.tiles_x + x);
            const unsigned long long t0 = warp_ns();
            unsigned v;
            while ((v = ld_acquire(sp)) == (unsigned)STAMP_PENDING) {
                if (warp_ns() - t0 > TMA_LIMIT_NS) {
                    set_status(st, EPIC_ERR_TIMEOUT);
                    gave_up = true;
                    break;
                }
            }
            written = lane < 8 && (int)v >= 0;
        }
    }
    if (any_written) *any_written = __any_sync(FULL, written);
    return !__any_sync(FULL, gave_up);
}

constexpr unsigned long long QUEUE_LIMIT_NS = 2000000000ull;  // 2 s

// Lane 0: the item of push p (pushes count from 0; the tickets after the
// sweep's take them in order), once pushed; -1 if none will come (nothing
// queued or being solved); -2 if a wait gave up (EPIC_ERR_TIMEOUT recorded)
// or another warp recorded an error.
__device__ int queue_wait(const BatchArgs &a, RunState *st, unsigned p) {
    const unsigned cap = (unsigned)a.total_tiles;
    const unsigned long long t0 = warp_ns();
    for (;;) {
        if (ld_acquire(&st->q_tail) > p) {
            // pushed: the value follows the ticket
            int *slot = a.relax_queue + p % cap;
            for (;;) {
                const int v = (int)ld_acquire(reinterpret_cast<const unsigned *>(slot));
                if (v >= 0) {
                    *(volatile int *)slot = -1;
                    return v;
                }
                if (warp_ns() - t0 > QUEUE_LIMIT_NS) {
                    set_status(st, EPIC_ERR_TIMEOUT);
                    return -2;
                }
            }
        }
        // q_busy counts every pushed item until its solve and pushes are
        // done, so when it reads 0 the tail read after it is final
        if (ld_acquire(reinterpret_cast<const unsigned *>(&st->q_busy)) == 0u &&
            ld_acquire(&st->q_tail) <= p)
            return -1;
        if (get_status(st) != 0) return -2;
        if (warp_ns() - t0 > QUEUE_LIMIT_NS) {
            set_status(st, EPIC_ERR_TIMEOUT);
            return -2;
        }
        __nanosleep(256);
    }
}

// Per-tile queue state (relax_queued): TILE_REQUESTED while the tile is
// queued, or while a solve of it has been asked for during its running solve
// (TILE_RUNNING), which then solves it again; 0 when idle.  So a tile is
// never solved by two warps at once, and a change next door is never lost.
constexpr int TILE_REQUESTED = 1, TILE_RUNNING = 2;

// Ask for a solve of tile nt (flat index): pushed if it is idle, else marked
// (queued already, or running: its warp solves it again).  Lane-local: called
// by the lane that watches nt.  Returns false if the slot wait gave up.
__device__ bool queue_push(const BatchArgs &a, RunState *st, int nt) {
    if (atomicOr(&a.relax_queued[nt], TILE_REQUESTED) != 0) return true;
    atomicAdd(&st->q_busy, 1);   // counted before it becomes visible
    const unsigned cap = (unsigned)a.total_tiles;
    const unsigned p = atomicAdd(&st->q_tail, 1u);
    int *slot = a.relax_queue + p % cap;
    // the slot's previous item (p - cap) may not have been taken yet
    const unsigned long long t0 = warp_ns();
    while (*(volatile int *)slot >= 0) {
        if (warp_ns() - t0 > QUEUE_LIMIT_NS) {
            set_status(st, EPIC_ERR_TIMEOUT);
            return false;
        }
    }
    __threadfence();
    *(volatile int *)slot = nt;
    return true;
}

// After tile (tx, ty) of pair P changed (rows `mod`, bit r = tile row r of
// rv; `edges` bit 0 / 1: column 0 / 63 changed in some row): lane k < 8
// asks for a solve of neighbour k if the change can border on it.  The tile's keys are written and fenced
// already.  Returns false in every lane if a push gave up.
__device__ bool queue_neighbours(const BatchArgs &a, int pi, RunState *st, int tx, int ty,
                                 int rv, unsigned long long mod, unsigned edges, int lane) {
    const PairDev &P = a.pairs[pi];
    bool ok = true;
    if (lane < 8) {
        const int dx = lane < 3 ? lane - 1 : lane < 5 ? 2 * lane - 7 : lane - 6;
        const int dy = lane < 3 ? -1 : lane < 5 ? 0 : 1;
        const int x = tx + dx, y = ty + dy;
        // a neighbour's ring holds the tile's border next to it: the top row
        // above, the bottom row below, column 0 (63) to the left (right),
        // and the corner pixels diagonally (whose change implies both)
        const bool rows = dy < 0 ? (mod & 2ull) != 0 : dy > 0 ? ((mod >> rv) & 1ull) != 0 : true;
        const bool cols = dx < 0 ? (edges & 1u) != 0 : dx > 0 ? (edges & 2u) != 0 : true;
        const bool near = rows && cols;
        if (near && x >= 0 && x < P.tiles_x && y >= 0 && y < P.tiles_y) {
            ok = queue_push(a, st, a.tile_base[pi] + y * P.tiles_x + x);
        }
    }
    return !__any_sync(FULL, !ok);
}

__device__ __forceinline__ int take_tile(unsigned *dispenser, int lane) {
    int t = 0;
    if (lane == 0) t = (int)atomicAdd(dispenser, 1u);
    return __shfl_sync(FULL, t, 0);
}

// One queue item: tile t (flat index; `sweep`: the item of the sweep),
// solved and solved again while a neighbour asked for it during the solve;
// then its completion is counted.  Returns false when the warp must leave (a wait gave up, or the
// run recorded an error).
template <int MAXR>
__device__ bool solve_item(const BatchArgs &a, RunState *st, WarpTile<MAXR> &T, int lane,
                           unsigned &phase, int t, bool sweep, unsigned long long item_cap) {
    const int pi = find_pair(a.tile_base, a.npairs, t);
    const PairDev &P = a.pairs[pi];
    const int lt = t - a.tile_base[pi];
    const int tx = lt % P.tiles_x, ty = lt / P.tiles_x;
    // phase 1 may still be writing the tile or its ring (no grid barrier
    // divides the phases); the sweep skips a tile whose neighbours were all
    // left unreached
    bool look = true;
    if (!wait_tile_and_ring(P, tx, ty, lane, st, sweep ? &look : nullptr)) return false;
    for (;;) {
        // running, not requested: from here on a change next door asks for
        // another solve.  A neighbour that found the tile queued or running
        // wrote its keys (and fenced them) before its atomic, so they are
        // visible after ours.
        if (lane == 0) {
            atomicExch(&a.relax_queued[t], TILE_RUNNING);
            __threadfence();
        }
        __syncwarp();
        if (look) {
            unsigned long long mod = 0;
            unsigned edges = 0;
            const int r = resolve_tile(P, lt, tx, ty, T, lane, phase, st, 1, &mod, &edges);
            if (r < 0) return false;
            if (r > 0 && !queue_neighbours(a, pi, st, tx, ty, tile_geo(P, tx, ty, lane).rv, mod,
                                           edges, lane))
                return false;
        }
        int again = 0;
        if (lane == 0) {
            again = atomicCAS(&a.relax_queued[t], TILE_RUNNING, 0) != TILE_RUNNING;
            atomicAdd(&st->q_items, 1u);
        }
        if (!__shfl_sync(FULL, again, 0)) break;
        look = true;
    }
    if (lane == 0) {
        __threadfence();   // this item's pushes before its completion
        atomicSub(&st->q_busy, 1);
        if (ld_acquire(&st->q_items) >= item_cap) set_status(st, EPIC_ERR_NOT_CONVERGED);
    }
    return get_status(st) == 0;
}

template <int MAXR>
__global__ void __launch_bounds__(RT_WARPS * 32) relax_kernel(const BatchArgs *__restrict__ ap) {
    const BatchArgs a = *ap;
    RunState *st = a.state;
    if (get_status(st) != 0) return;  // same decision in every CTA
    // a launch replayed for a smaller batch may have more CTAs than tile
    // workers need: the extra CTAs leave at once and the barrier counts only
    // the others
    const unsigned nblocks =
        min(gridDim.x, (unsigned)((a.total_tiles + RT_WARPS - 1) / RT_WARPS));
    if (blockIdx.x >= nblocks) return;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    WarpTile<MAXR> &T = reinterpret_cast<WarpTile<MAXR> *>(smem)[threadIdx.x >> 5];
    unsigned phase = 0;   // parity of the warp's mbarrier
    if (lane == 0) {
        const unsigned bar = (unsigned)__cvta_generic_to_shared(&T.bar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    // phase 1, in two halves handed out by one counter: index u < T is tile
    // u of the first half (tx + ty even), index T + u tile u of the second.
    // Every first-half tile is taken before any second-half tile, so a
    // second-half tile only waits (bounded) for its four edge neighbours,
    // each already held by a running warp; no grid barrier divides the
    // halves.
    for (int u = take_tile(&st->work[3], lane); u < 2 * a.total_tiles;
         u = take_tile(&st->work[3], lane)) {
        const int half = u >= a.total_tiles;
        const int t = u - (half ? a.total_tiles : 0);
        const int pi = find_pair(a.tile_base, a.npairs, t);
        const PairDev &P = a.pairs[pi];
        const int lt = t - a.tile_base[pi];
        const int tx = lt % P.tiles_x, ty = lt / P.tiles_x;
        if (((tx + ty) & 1) != half) continue;
        if (half && !wait_edge_neighbours(P, tx, ty, lane, st)) return;
        if (!fresh_tile(P, lt, tx, ty, T, lane, phase, st, half == 1)) return;
    }

    // phase 2: a work queue of tiles whose ring may have changed.  Ticket
    // h < T (the tile count) is tile h, the initial sweep; later tickets
    // take the tiles pushed since, in order.  A tile whose keys change
    // pushes the neighbours its changed rows border on (unless they are
    // already queued), and is pushed again itself if a neighbour changes
    // while it is being solved.  q_busy counts the items pushed (or of the
    // sweep) that are not finished; a warp whose ticket has no item while
    // q_busy is 0 knows that none will come, since only the solve of an
    // unfinished item pushes.  So the phase needs no grid barrier: a front
    // of changes runs on through the tiles as soon as each is solved.
    const int Tt = a.total_tiles;
    const unsigned long long item_cap = (unsigned long long)a.max_passes * (unsigned)Tt;
    // the sweep hands out `chunk` consecutive tiles per ticket while that
    // leaves every warp several tickets (fewer counter atomics, and a chunk's
    // tiles solved in turn see each other's results)
    const int chunk = max(1, min(SCAN_CHUNK, Tt / (4 * (int)nblocks * RT_WARPS)));
    const unsigned n0 = (unsigned)((Tt + chunk - 1) / chunk);   // tickets of the sweep
    for (;;) {
        unsigned h = 0;
        if (lane == 0) h = atomicAdd(&st->q_head, 1u);
        h = __shfl_sync(FULL, h, 0);
        if (h < n0) {
            for (int q = 0; q < chunk && (int)h * chunk + q < Tt; ++q)
                if (!solve_item(a, st, T, lane, phase, (int)h * chunk + q, true, item_cap))
                    return;
        } else {
            // wait for the ticket's item, or for the end of the work
            int got = -1;
            if (lane == 0) got = queue_wait(a, st, h - n0);
            got = __shfl_sync(FULL, got, 0);
            if (got == -2) return;   // a wait gave up or another warp failed
            if (got < 0) break;      // no item will come
            if (!solve_item(a, st, T, lane, phase, got, true, item_cap)) return;
        }
    }
    // every item is finished: report the re-solves as equivalent passes
    if (lane == 0) {
        const unsigned items = ld_acquire(&st->q_items);
        st->passes = 1 + (int)(((unsigned long long)items - (unsigned)Tt + (unsigned)Tt - 1) /
                               (unsigned)Tt);
    }
}

}  // namespace

size_t relax_smem_bytes(int max_rows) {
    return RT_WARPS * (max_rows <= 8    ? sizeof(WarpTile<8>)
                       : max_rows <= 16 ? sizeof(WarpTile<16>)
                                        : sizeof(WarpTile<32>));
}

cudaError_t launch_relax(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc,
                         int max_rows, bool fixed_grid, int *grid_used) {
    if (max_rows < 1 || max_rows > 32) return cudaErrorInvalidValue;
    // instances for tile heights up to 8, 16 and 32: the smaller the tile,
    // the less shared memory a warp holds and the more warps share an SM
    void (*kernel)(const BatchArgs *) = max_rows <= 8    ? relax_kernel<8>
                                        : max_rows <= 16 ? relax_kernel<16>
                                                         : relax_kernel<32>;
    const size_t smem = relax_smem_bytes(max_rows);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, RT_WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * lc.num_sms;
    const int need = (a.total_tiles + RT_WARPS - 1) / RT_WARPS;
    if (!fixed_grid && grid > need) grid = need;
    if (grid < 1) grid = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(RT_WARPS * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = lc.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (grid_used) *grid_used = grid;
    return cudaLaunchKernelEx(&cfg, kernel, dev);
}

}  // namespace epic
