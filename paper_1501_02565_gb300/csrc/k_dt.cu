// Stage (a): geodesic assignment map L and distance D (Sec. 3.4 "Geodesic
// Voronoi diagram"; D_G of Eq. 3 on the 8-connected grid).
//
// Each pixel's packed key (D, L) is the minimum over all matches m and all
// grid paths from p_m of (path cost, m), with path costs summed exactly in
// fixed point (units of 2^-31) from the steps |p-q| (C(p)+C(q))/2.  Any
// order of relaxation steps that ends when no step improves any key reaches
// these keys bit for bit: with exact sums every prefix of an optimal path is
// optimal, so a state that no single step improves is the minimum.  The
// kernel exploits that freedom:
//
//   phase 1  every tile is solved alone in shared memory on its region
//            (tile + apron + 1-px ring), with the seeds of that region, and
//            writes its tile's keys;
//   phase 2  repeated passes: a tile whose border can be improved from the
//            current keys of the pixels just outside it reloads
//            (tile + ring) and re-solves; the passes end when no tile is
//            dirty, i.e. no step improves any key anywhere.  Every tile
//            records the last pass that wrote it; a tile is checked in pass k
//            only if one of its eight neighbours was written in pass k-1 or
//            later (phase 1 counts as pass 0), because a tile checked clean
//            stays clean until a neighbour changes.
//
// The in-tile solver runs directional sweeps (down, up, right, left), each
// relaxing a pixel from its three neighbours on the side the sweep comes
// from; a warp sweeps 32 adjacent lines in lock step.  One kernel launch
// holds all passes: it is a cooperative launch (all CTAs co-resident) and the
// passes are separated by a grid barrier whose wait is bounded in time.
#include "epic_internal.cuh"

namespace epic {

namespace {

// Shared-memory solve region.  Region cell (c, r) is image pixel
// (x0 + c, y0 + r); row pitch P is odd so that a warp reading one column
// (32 rows) of 8-byte keys touches every bank pair once.
struct Region {
    int x0, y0, RW, RH, P;
    int bx0, bx1, by0, by1;  // updatable cells: interior and inside the image
};

__device__ __forceinline__ int odd_pitch(int w) { return w | 1; }

__device__ __forceinline__ Region make_region(const PairDev &P, int gx0,
                                              int gy0, int tw, int th,
                                              int apron) {
    Region g;
    g.x0 = gx0 - apron - 1;
    g.y0 = gy0 - apron - 1;
    g.RW = tw + 2 * apron + 2;
    g.RH = th + 2 * apron + 2;
    g.P = odd_pitch(g.RW);
    g.bx0 = max(1, -g.x0);
    g.bx1 = min(g.RW - 2, P.W - 1 - g.x0);
    g.by0 = max(1, -g.y0);
    g.by1 = min(g.RH - 2, P.H - 1 - g.y0);
    return g;
}

// Best of the current key and the three candidates reached from the
// neighbours at offsets ax (axis step) and d1, d2 (diagonal steps).
__device__ __forceinline__ int relax3(pkey_t *K, const unsigned *h, int idx,
                                      int ax, int d1, int d2) {
    const pkey_t kp = K[idx];
    const unsigned hp = h[idx];
    pkey_t best = kp;
    pkey_t c = step_key(K[idx + ax], step_axis(hp, h[idx + ax]));
    best = c < best ? c : best;
    c = step_key(K[idx + d1], step_diag(hp, h[idx + d1]));
    best = c < best ? c : best;
    c = step_key(K[idx + d2], step_diag(hp, h[idx + d2]));
    best = c < best ? c : best;
    if (best < kp) {
        K[idx] = best;
        return 1;
    }
    return 0;
}

// Sweep the region to its fixed point.  Returns 1 if any key changed.
//
// Sweep schedule: a vertical sweep runs down (or up) every column of the
// region, a horizontal one along every row.  With whole = 0 each line is cut
// into segments so that all threads of the CTA have a segment (more threads
// busy, but a key crosses one segment boundary per iteration); with whole = 1
// a thread runs whole lines (fewer threads busy, fewer iterations).  A
// thread takes work items (column or row segments) with a stride of the
// CTA size, so regions with more lines than threads are covered too; lanes
// of a warp step through adjacent lines together.  Any schedule reaches the
// same fixed point.
__device__ int local_solve(pkey_t *K, const unsigned *h, const Region &g,
                           RunState *st, int whole) {
    const int ncols = g.bx1 - g.bx0 + 1, nrows = g.by1 - g.by0 + 1;
    if (ncols <= 0 || nrows <= 0) return 0;
    const int T = blockDim.x, tid = threadIdx.x, P = g.P;
    const int nsegV = whole ? 1 : max(1, T / ncols);
    const int segV = (nrows + nsegV - 1) / nsegV;
    const int itemsV = ncols * nsegV, roundsV = (itemsV + T - 1) / T;
    const int nsegH = whole ? 1 : max(1, T / nrows);
    const int segH = (ncols + nsegH - 1) / nsegH;
    const int itemsH = nrows * nsegH, roundsH = (itemsH + T - 1) / T;

    // Sweeps run in the cyclic order down, up, right, left.  The region is
    // at its fixed point once four consecutive sweeps (one per direction,
    // hence every pixel against all eight neighbours) changed nothing, which
    // can happen in the middle of a cycle.
    const int cap = 4 * g.RW * g.RH;  // Bellman-Ford bound on useful sweeps
    int any = 0, quiet = 0;
    for (int sw = 0; sw < cap; ++sw) {
        const int dir = sw & 3;
        int ch = 0;
        if (dir < 2) {
            // down (dir 0): from the row above; up (dir 1): from the row below
            const int off = dir == 0 ? -P : P;
            for (int rv = 0; rv < roundsV; ++rv) {
                const int w = tid + rv * T;
                const bool vu = w < itemsV;
                const int vx = g.bx0 + w % ncols;
                const int vy0 = g.by0 + (w / ncols) * segV;
                const int vy1 = min(g.by1, vy0 + segV - 1);
                for (int s = 0; s < segV; ++s) {
                    const int y = dir == 0 ? vy0 + s : vy1 - s;
                    if (vu && y >= vy0 && y <= vy1)
                        ch |= relax3(K, h, y * P + vx, off, off - 1, off + 1);
                    __syncwarp();
                }
            }
        } else {
            // right (dir 2): from the column on the left; left (dir 3): from
            // the column on the right
            const int off = dir == 2 ? -1 : 1;
            for (int rh = 0; rh < roundsH; ++rh) {
                const int w = tid + rh * T;
                const bool hu = w < itemsH;
                const int hy = g.by0 + w % nrows;
                const int hx0 = g.bx0 + (w / nrows) * segH;
                const int hx1 = min(g.bx1, hx0 + segH - 1);
                for (int s = 0; s < segH; ++s) {
                    const int x = dir == 2 ? hx0 + s : hx1 - s;
                    if (hu && x >= hx0 && x <= hx1)
                        ch |= relax3(K, h, hy * P + x, off, off - P, off + P);
                    __syncwarp();
                }
            }
        }
        if (__syncthreads_or(ch)) {
            any = 1;
            quiet = 0;
        } else if (++quiet == 4) {
            return any;
        }
    }
    if (tid == 0) set_status(st, EPIC_ERR_NOT_CONVERGED);
    return any;
}

// TMA staging: one mbarrier per CTA; every use is separated from the next by
// __syncthreads, and all threads track its phase in `phase`.
struct Tma {
    unsigned mbar;   // shared-space address of the barrier
    unsigned phase;
};

__device__ __forceinline__ void tma_init(Tma &t, unsigned long long *bar) {
    t.mbar = (unsigned)__cvta_generic_to_shared(bar);
    t.phase = 0;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(t.mbar) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
}

// Thread 0 starts a 2D tensor copy of `bytes` bytes at (x, y) into `dst`.
__device__ __forceinline__ void tma_load_2d(const Tma &t, const CUtensorMap *map, void *dst,
                                            int x, int y, unsigned bytes) {
    if (threadIdx.x != 0) return;
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(t.mbar), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(d),
        "l"(map), "r"(x), "r"(y), "r"(t.mbar)
        : "memory");
}

// All threads wait for the copy, at most TMA_LIMIT_NS; on time-out the run
// reports EPIC_ERR_TIMEOUT.  Returns, in every thread of the CTA, whether
// the copy completed for all of them (false if any thread gave up).
constexpr unsigned long long TMA_LIMIT_NS = 1000000000ull;
__device__ __forceinline__ bool tma_wait(Tma &t, RunState *st,
                                         unsigned long long limit_ns = TMA_LIMIT_NS) {
    const unsigned long long t0 = global_ns();
    int gave_up = 0;
    for (;;) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
            " selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(t.mbar), "r"(t.phase)
            : "memory");
        if (done) break;
        if (global_ns() - t0 > limit_ns) {
            set_status(st, EPIC_ERR_TIMEOUT);
            gave_up = 1;
            break;
        }
    }
    t.phase ^= 1u;
    return __syncthreads_or(gave_up) == 0;
}

// Half-costs of the region in fixed-point units; a cost outside [0, C_MAX)
// (or not finite) is an invalid input.  With TMA the region's costs are
// first copied as one box into `stage` (free shared memory, 128-byte
// aligned), from the region's x origin rounded down to a multiple of 4;
// cells outside the image are filled with zeros by the copy and get h = 0
// here, as on the plain path.  Returns false (in every thread) when the
// copy's wait timed out: the stage is then not read, and the caller leaves
// the kernel (the run has recorded EPIC_ERR_TIMEOUT; the copy may still land
// in this CTA's shared memory after it has left).
__device__ __forceinline__ bool load_costs(const PairDev &P, const Region &g,
                                           unsigned *h, RunState *st, bool fresh,
                                           float *stage, Tma &tma) {
    bool bad = false;
    if (P.tma_cost) {
        const int bw = fresh ? P.tma_bw_fresh : P.tma_bw_again;
        const int xa = g.x0 - (((g.x0 % 4) + 4) % 4);
        tma_load_2d(tma, fresh ? &P.tm_cost_fresh : &P.tm_cost_again, stage, xa, g.y0,
                    (unsigned)(bw * g.RH * 4));
        if (!tma_wait(tma, st)) return false;
        const int off = g.x0 - xa;
        for (int i = threadIdx.x; i < g.RW * g.RH; i += blockDim.x) {
            int r = i / g.RW, c = i - r * g.RW;
            int gx = g.x0 + c, gy = g.y0 + r;
            bool in = gx >= 0 && gx < P.W && gy >= 0 && gy < P.H;
            h[r * g.P + c] = in ? half_cost(stage[r * bw + c + off], &bad) : 0u;
        }
        __syncthreads();   // the stage area is reused by the caller
    } else {
        for (int i = threadIdx.x; i < g.RW * g.RH; i += blockDim.x) {
            int r = i / g.RW, c = i - r * g.RW;
            int gx = g.x0 + c, gy = g.y0 + r;
            bool in = gx >= 0 && gx < P.W && gy >= 0 && gy < P.H;
            h[r * g.P + c] = in ? half_cost(__ldg(P.C + (size_t)gy * P.W + gx), &bad) : 0u;
        }
    }
    if (bad) set_status(st, EPIC_ERR_INVALID);
    return true;
}

// The relaxation's shared memory: keys (RH x P), half-costs (RH x P); the
// key area doubles as the TMA stage for the costs, which are converted
// before the keys are written.
__device__ __forceinline__ float *stage_area(unsigned char *smem) {
    return reinterpret_cast<float *>(((uintptr_t)smem + 127) & ~(uintptr_t)127);
}

// A key as written back: with a cap map (the exact variant's single-source
// runs), a distance beyond the pixel's cap is left unreached, so the run
// stops spreading where it can no longer matter.  The cap is 1-Lipschitz in
// the same fixed-point metric, so every pixel on a shortest path to a
// pixel within its cap is within its own cap: capped runs are exact there.
__device__ __forceinline__ pkey_t capped(const PairDev &P, size_t p, pkey_t k) {
    return P.cap && key_dunits(k) > key_dunits(P.cap[p]) ? KEY_INF : k;
}

// The pair a flat tile index belongs to (a division when all pairs have the
// same tile count, as the exact variant's single-source pseudo-pairs do).
__device__ __forceinline__ int tile_pair(const BatchArgs &a, int t) {
    return a.uniform_tiles > 0 ? t / a.uniform_tiles : find_pair(a.tile_base, a.npairs, t);
}

// Phase 1: solve tile (tx, ty) on its region from its seeds alone.  Returns
// false when the cost staging timed out (the CTA must leave the kernel).
__device__ bool solve_fresh(const PairDev &P, int tx, int ty, pkey_t *K,
                            unsigned *h, RunState *st, float *stage, Tma &tma) {
    const int gx0 = tx * P.tile_w, gy0 = ty * P.tile_h;
    const Region g = make_region(P, gx0, gy0, P.tile_w, P.tile_h, P.apron);
    // seeds: the region lies within the 3x3 tiles around (tx, ty)
    const int ctx0 = max(0, g.x0) / P.tile_w;
    const int ctx1 = min(P.W - 1, g.x0 + g.RW - 1) / P.tile_w;
    const int cty0 = max(0, g.y0) / P.tile_h;
    const int cty1 = min(P.H - 1, g.y0 + g.RH - 1) / P.tile_h;
    int nseeds = 0;
    for (int cy = cty0; cy <= cty1; ++cy)
        for (int cx = ctx0; cx <= ctx1; ++cx) {
            const int t = cy * P.tiles_x + cx;
            nseeds += P.tile_start[t + 1] - P.tile_start[t];
        }
    if (nseeds == 0) {
        // no seed near the tile (the single-source runs of the exact variant
        // have one in the whole image): it stays unreached until the
        // verification passes bring distances in from its neighbours.  Its
        // stamp says "never written", so its neighbours (unreached too, if
        // also seedless) skip the border test in the first pass
        if (threadIdx.x == 0) P.tile_stamp[ty * P.tiles_x + tx] = -1;
        for (int i = threadIdx.x; i < P.tile_w * P.tile_h; i += blockDim.x) {
            const int ly = i / P.tile_w, lx = i - ly * P.tile_w;
            const int gx = gx0 + lx, gy = gy0 + ly;
            if (gx < P.W && gy < P.H) P.keys[(size_t)gy * P.W + gx] = KEY_INF;
        }
        __syncthreads();
        return true;
    }
    if (!load_costs(P, g, h, st, true, stage, tma)) return false;
    for (int i = threadIdx.x; i < g.RW * g.RH; i += blockDim.x) {
        int r = i / g.RW, c = i - r * g.RW;
        K[r * g.P + c] = KEY_INF;
    }
    __syncthreads();
    for (int cy = cty0; cy <= cty1; ++cy) {
        for (int cx = ctx0; cx <= ctx1; ++cx) {
            int t = cy * P.tiles_x + cx;
            int s0 = P.tile_start[t], s1 = P.tile_start[t + 1];
            for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
                int m = P.tile_seeds[s];
                float4 mt = __ldg(P.matches + m);
                int px = (int)floorf(mt.x + 0.5f) - g.x0;
                int py = (int)floorf(mt.y + 0.5f) - g.y0;
                if (px >= 0 && px < g.RW && py >= 0 && py < g.RH)
                    atomicMin(&K[py * g.P + px],
                              make_key(P.seed_init ? P.seed_init[m] : 0ull, (unsigned)m));
            }
        }
    }
    __syncthreads();
    local_solve(K, h, g, st, P.sweep);
    // write the tile's own pixels and mark it written in pass 0
    if (threadIdx.x == 0) P.tile_stamp[ty * P.tiles_x + tx] = 0;
    const int off = P.apron + 1;
    for (int i = threadIdx.x; i < P.tile_w * P.tile_h; i += blockDim.x) {
        int ly = i / P.tile_w, lx = i - ly * P.tile_w;
        int gx = gx0 + lx, gy = gy0 + ly;
        if (gx < P.W && gy < P.H)
            P.keys[(size_t)gy * P.W + gx] =
                capped(P, (size_t)gy * P.W + gx, K[(ly + off) * g.P + lx + off]);
    }
    __syncthreads();
    return true;
}

__device__ __forceinline__ pkey_t ld_key(const pkey_t *p) { return __ldcg(p); }

// Can a border pixel of the tile be improved by a step from a pixel outside
// it?  Keys of other tiles may be rewritten during the launch, so they are
// read through L2 (ld.global.cg), never from a stale L1 line.
__device__ bool border_dirty(const PairDev &P, int tx, int ty) {
    const int gx0 = tx * P.tile_w, gy0 = ty * P.tile_h;
    const int gx1 = min(P.W - 1, gx0 + P.tile_w - 1);
    const int gy1 = min(P.H - 1, gy0 + P.tile_h - 1);
    const int w = gx1 - gx0 + 1, hgt = gy1 - gy0 + 1;
    const int n_top = w, n_bot = hgt > 1 ? w : 0;
    const int n_side = max(0, hgt - 2);
    const int n_left = n_side, n_right = w > 1 ? n_side : 0;
    const int total = n_top + n_bot + n_left + n_right;
    int dirty = 0;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        int x, y;
        if (i < n_top) { x = gx0 + i; y = gy0; }
        else if (i < n_top + n_bot) { x = gx0 + (i - n_top); y = gy1; }
        else if (i < n_top + n_bot + n_left) { x = gx0; y = gy0 + 1 + (i - n_top - n_bot); }
        else { x = gx1; y = gy0 + 1 + (i - n_top - n_bot - n_left); }
        const size_t p = (size_t)y * P.W + x;
        const pkey_t kp = ld_key(P.keys + p);
        bool bad = false;
        const unsigned hp = half_cost(__ldg(P.C + p), &bad);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int dx = (k == 0 || k == 4 || k == 6) ? 1 : (k == 1 || k == 5 || k == 7) ? -1 : 0;
            const int dy = (k == 2 || k == 4 || k == 5) ? 1 : (k == 3 || k == 6 || k == 7) ? -1 : 0;
            const int qx = x + dx, qy = y + dy;
            if (qx < 0 || qx >= P.W || qy < 0 || qy >= P.H) continue;
            if (qx >= gx0 && qx <= gx1 && qy >= gy0 && qy <= gy1) continue;
            const size_t q = (size_t)qy * P.W + qx;
            const pkey_t kq = ld_key(P.keys + q);
            const unsigned hq = half_cost(__ldg(P.C + q), &bad);
            const unsigned long long w = (dx != 0 && dy != 0) ? step_diag(hp, hq) : step_axis(hp, hq);
            // an improvement beyond the pixel's cap would be written back
            // unreached, so it does not make the tile dirty
            dirty |= capped(P, p, step_key(kq, w)) < kp;
        }
    }
    return __syncthreads_or(dirty) != 0;
}

// Phase 2 re-solve of tile (tx, ty) from the current keys (tile + ring).
// Returns 1 if any key of the region changed, 0 if none did, -1 if the cost
// staging timed out (the CTA must leave the kernel); the same in every
// thread.
__device__ int solve_again(const PairDev &P, int tx, int ty, pkey_t *K,
                            unsigned *h, RunState *st, int pass, float *stage, Tma &tma) {
    const int gx0 = tx * P.tile_w, gy0 = ty * P.tile_h;
    const Region g = make_region(P, gx0, gy0, P.tile_w, P.tile_h, 0);
    if (!load_costs(P, g, h, st, false, stage, tma)) return -1;
    for (int i = threadIdx.x; i < g.RW * g.RH; i += blockDim.x) {
        int r = i / g.RW, c = i - r * g.RW;
        int gx = g.x0 + c, gy = g.y0 + r;
        bool in = gx >= 0 && gx < P.W && gy >= 0 && gy < P.H;
        K[r * g.P + c] = in ? ld_key(P.keys + (size_t)gy * P.W + gx) : KEY_INF;
    }
    __syncthreads();
    const bool changed = local_solve(K, h, g, st, P.sweep) != 0;
    if (changed) {
        for (int i = threadIdx.x; i < P.tile_w * P.tile_h; i += blockDim.x) {
            int ly = i / P.tile_w, lx = i - ly * P.tile_w;
            int gx = gx0 + lx, gy = gy0 + ly;
            if (gx < P.W && gy < P.H)
                P.keys[(size_t)gy * P.W + gx] =
                    capped(P, (size_t)gy * P.W + gx, K[(ly + 1) * g.P + lx + 1]);
        }
    }
    if (threadIdx.x == 0) P.tile_stamp[ty * P.tiles_x + tx] = pass;
    __syncthreads();
    return changed ? 1 : 0;
}

// Chunked passes: queue the eight neighbours of tile t (flat index; local
// (tx, ty) in pair pi) for pass `next`, each at most once (threads 0-7).
__device__ __forceinline__ void queue_neighbours(const BatchArgs &a, RunState *st, int pi,
                                                 int tx, int ty, int next) {
    if (threadIdx.x >= 8) return;
    const PairDev &P = a.pairs[pi];
    const int k = threadIdx.x;
    const int x = tx + (k < 3 ? k - 1 : k < 5 ? 2 * k - 7 : k - 6);
    const int y = ty + (k < 3 ? -1 : k < 5 ? 0 : 1);
    if (x < 0 || x >= P.tiles_x || y < 0 || y >= P.tiles_y) return;
    const int nt = a.tile_base[pi] + y * P.tiles_x + x;
    if (atomicMax(a.wl_queued + nt, next + 1) < next + 1) {
        const unsigned q = atomicAdd(&st->wl_count[next % 3], 1u);
        a.wl[(size_t)(next % 3) * a.total_tiles + q] = nt;
    }
}

// CHUNKED: how the verification passes hand out tiles.  false (the
// interpolator's runs: a handful of passes, about half of the tiles
// re-solved in the first): one tile at a time.  true (the single-source runs
// of the exact variant: dozens of passes while distances cross the image
// tile by tile, each re-solving a thin front): chunks of tiles whose
// neighbour stamps are read in parallel.  The chunked loop keeps more state
// and, at the four-CTA register budget, costs the interpolator's sweeps a
// spill (2.21 -> 2.33 ms); the single-source runs go 3.1 -> 2.1 s per pair.
template <bool CHUNKED>
__global__ void __launch_bounds__(DT_THREADS) dt_kernel(const BatchArgs *__restrict__ ap) {
    const BatchArgs a = *ap;
    extern __shared__ __align__(16) unsigned char smem[];
    RunState *st = a.state;
    if (get_status(st) != 0) return;  // same decision in every CTA
    // a launch replayed for a smaller batch may have more CTAs than tiles:
    // the extra CTAs leave at once and the barrier counts only the others
    const unsigned nblocks = min(gridDim.x, (unsigned)a.total_tiles);
    if (blockIdx.x >= nblocks) return;
    __shared__ int s_pair, s_local, s_tile;
    __shared__ __align__(8) unsigned long long s_bar;
    Tma tma;
    tma_init(tma, &s_bar);
    float *stage = stage_area(smem);
    // tiles are handed out one at a time from a counter, so that CTAs whose
    // tiles converge quickly take more of them
    auto next_tile = [&](unsigned *dispenser) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int t = (int)atomicAdd(dispenser, 1u);
            s_tile = t;
            if (t < a.total_tiles) {
                s_pair = tile_pair(a, t);
                s_local = t - a.tile_base[s_pair];
            }
        }
        __syncthreads();
        return s_tile;
    };

    // phase 1
    for (int t = next_tile(&st->work[3]); t < a.total_tiles; t = next_tile(&st->work[3])) {
        const PairDev &P = a.pairs[s_pair];
        const Region g = make_region(P, 0, 0, P.tile_w, P.tile_h, P.apron);
        pkey_t *K = reinterpret_cast<pkey_t *>(smem);
        unsigned *h = reinterpret_cast<unsigned *>(smem + sizeof(pkey_t) * g.RH * g.P);
        if (!solve_fresh(P, s_local % P.tiles_x, s_local / P.tiles_x, K, h, st, stage, tma))
            return;
    }
    if (!grid_sync(st, nblocks)) return;

    // phase 2
    for (int pass = 0;; ++pass) {
        if (pass >= a.max_passes) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                set_status(st, EPIC_ERR_NOT_CONVERGED);
                st->passes = pass;
            }
            return;
        }
        unsigned *cnt = &st->changed[pass % 3];
        unsigned *disp = &st->work[pass % 3];
        if constexpr (!CHUNKED) {
            for (int t = next_tile(disp); t < a.total_tiles; t = next_tile(disp)) {
                const PairDev &P = a.pairs[s_pair];
                const int tx = s_local % P.tiles_x, ty = s_local / P.tiles_x;
                // threads 0-7 read the eight neighbour stamps at once
                bool nb = false;
                if (threadIdx.x < 8) {
                    const int k = threadIdx.x;
                    const int x = tx + (k < 3 ? k - 1 : k < 5 ? 2 * k - 7 : k - 6);
                    const int y = ty + (k < 3 ? -1 : k < 5 ? 0 : 1);
                    nb = x >= 0 && x < P.tiles_x && y >= 0 && y < P.tiles_y &&
                         __ldcg(P.tile_stamp + y * P.tiles_x + x) >= pass;
                }
                if (__syncthreads_or(nb) && border_dirty(P, tx, ty)) {
                    const Region g = make_region(P, 0, 0, P.tile_w, P.tile_h, 0);
                    pkey_t *K = reinterpret_cast<pkey_t *>(smem);
                    unsigned *h = reinterpret_cast<unsigned *>(smem + sizeof(pkey_t) * g.RH * g.P);
                    if (solve_again(P, tx, ty, K, h, st, pass + 1, stage, tma) < 0) return;
                    if (threadIdx.x == 0) atomicAdd(cnt, 1u);
                }
                __syncthreads();
            }
        } else {
            // Pass 0 scans every tile, PASS_CHUNK at a time: the first
            // 8 x PASS_CHUNK threads read the chunk's neighbour stamps in
            // parallel and flag the tiles with a neighbour written since phase
            // 1; only those go on to the border test.  A tile that changes
            // queues its eight neighbours for the next pass, and every later
            // pass works through that list alone (a single-source run
            // re-solves a thin front, and scanning every tile in each of its
            // dozen passes cost more than the re-solves).  The loop state
            // lives in shared memory, so nothing extra stays in registers
            // across a re-solve.
            __shared__ int s_t0, s_bits;
            if (pass == 0) {
                for (;;) {
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        s_t0 = (int)atomicAdd(disp, (unsigned)PASS_CHUNK);
                        s_bits = 0;
                    }
                    __syncthreads();
                    if (s_t0 >= a.total_tiles) break;
                    if (threadIdx.x < 8 * PASS_CHUNK) {
                        const int t = s_t0 + (threadIdx.x >> 3), k = threadIdx.x & 7;
                        if (t < a.total_tiles) {
                            const int pi = tile_pair(a, t);
                            const PairDev &P = a.pairs[pi];
                            const int lt = t - a.tile_base[pi];
                            const int x = lt % P.tiles_x + (k < 3 ? k - 1 : k < 5 ? 2 * k - 7 : k - 6);
                            const int y = lt / P.tiles_x + (k < 3 ? -1 : k < 5 ? 0 : 1);
                            if (x >= 0 && x < P.tiles_x && y >= 0 && y < P.tiles_y &&
                                __ldcg(P.tile_stamp + y * P.tiles_x + x) >= pass)
                                atomicOr(&s_bits, 1 << (threadIdx.x >> 3));
                        }
                    }
                    for (;;) {
                        __syncthreads();
                        if (threadIdx.x == 0) {
                            const int b = s_bits;
                            if (b) {
                                const int t = s_t0 + __ffs(b) - 1;
                                s_bits = b & (b - 1);
                                s_tile = t;
                                s_pair = tile_pair(a, t);
                                s_local = t - a.tile_base[s_pair];
                            } else {
                                s_tile = -1;
                            }
                        }
                        __syncthreads();
                        if (s_tile < 0) break;
                        const PairDev &P = a.pairs[s_pair];
                        const int tx = s_local % P.tiles_x, ty = s_local / P.tiles_x;
                        if (border_dirty(P, tx, ty)) {
                            const Region g = make_region(P, 0, 0, P.tile_w, P.tile_h, 0);
                            pkey_t *K = reinterpret_cast<pkey_t *>(smem);
                            unsigned *h = reinterpret_cast<unsigned *>(smem + sizeof(pkey_t) * g.RH * g.P);
                            const int r = solve_again(P, tx, ty, K, h, st, pass + 1, stage, tma);
                            if (r < 0) return;
                            if (r > 0) queue_neighbours(a, st, s_pair, tx, ty, pass + 1);
                            if (threadIdx.x == 0) atomicAdd(cnt, 1u);
                        }
                    }
                }
            } else {
                // the list of this pass was complete before the last barrier
                const unsigned n = ld_acquire(&st->wl_count[pass % 3]);
                const int *list = a.wl + (size_t)(pass % 3) * a.total_tiles;
                for (;;) {
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        const unsigned q = atomicAdd(disp, 1u);
                        s_tile = q < n ? list[q] : -1;
                        if (s_tile >= 0) {
                            s_pair = tile_pair(a, s_tile);
                            s_local = s_tile - a.tile_base[s_pair];
                        }
                    }
                    __syncthreads();
                    if (s_tile < 0) break;
                    const PairDev &P = a.pairs[s_pair];
                    const int tx = s_local % P.tiles_x, ty = s_local / P.tiles_x;
                    if (border_dirty(P, tx, ty)) {
                        const Region g = make_region(P, 0, 0, P.tile_w, P.tile_h, 0);
                        pkey_t *K = reinterpret_cast<pkey_t *>(smem);
                        unsigned *h = reinterpret_cast<unsigned *>(smem + sizeof(pkey_t) * g.RH * g.P);
                        const int r = solve_again(P, tx, ty, K, h, st, pass + 1, stage, tma);
                        if (r < 0) return;
                        if (r > 0) queue_neighbours(a, st, s_pair, tx, ty, pass + 1);
                        if (threadIdx.x == 0) atomicAdd(cnt, 1u);
                    }
                }
            }
        }
        if (!grid_sync(st, nblocks)) return;
        const unsigned dirty = ld_acquire(cnt);
        // the counters of pass-1 (== pass+2 mod 3) were last used before
        // this barrier; clear them for pass+2
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->changed[(pass + 2) % 3] = 0;
            st->work[(pass + 2) % 3] = 0;
            st->wl_count[(pass + 2) % 3] = 0;
        }
        if (dirty == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) st->passes = pass + 1;
            return;
        }
    }
}

// Self-test of the bounded waits (failure detection without a GPU fault):
// one CTA waits for a second CTA that does not exist at the grid barrier
// (which = 0), or for a TMA transaction that is never issued on an
// mbarrier (which = 1).  Either wait must give up after limit_ns and record
// EPIC_ERR_TIMEOUT, leaving the context usable.
__global__ void wait_selftest_kernel(RunState *st, int which, unsigned long long limit_ns) {
    if (which == 0) {
        grid_sync(st, 2u, limit_ns);
    } else {
        __shared__ __align__(8) unsigned long long bar;
        Tma t;
        tma_init(t, &bar);
        tma_wait(t, st, limit_ns);
    }
}

}  // namespace

cudaError_t launch_wait_selftest(RunState *st, int which, unsigned long long limit_ns,
                                 cudaStream_t stream) {
    wait_selftest_kernel<<<1, 32, 0, stream>>>(st, which, limit_ns);
    return cudaGetLastError();
}

size_t dt_smem_bytes(int tile_w, int tile_h, int apron) {
    int RW = tile_w + 2 * apron + 2, RH = tile_h + 2 * apron + 2;
    int P = RW | 1;
    // keys and half-costs, plus alignment slack for the TMA stage; the stage
    // (RH x (RW + 6) floats at most) fits in the key area (RH x P x 8 bytes)
    return (size_t)RH * P * (sizeof(pkey_t) + sizeof(unsigned)) + 128;
}

cudaError_t launch_dt(const BatchArgs &a, const BatchArgs *dev, const LaunchCfg &lc,
                      int max_tile_w, int max_tile_h, int max_apron, bool fixed_grid,
                      int *grid_used, bool chunked_passes) {
    size_t smem = dt_smem_bytes(max_tile_w, max_tile_h, max_apron);
    void (*kernel)(const BatchArgs *) = chunked_passes ? dt_kernel<true> : dt_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(
        kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel,
                                                      DT_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * lc.num_sms;
    if (!fixed_grid && grid > a.total_tiles) grid = a.total_tiles;
    if (grid < 1) grid = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(DT_THREADS);
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
