// k_fused.cu -- the fused, temporally blocked 2D path: one launch advances the
// field AND the growth cones K steps (rows a1-a6) with one HBM/L2 round trip
// of the field.
//
// Each CTA owns an interior tile of TX x TY nodes.  It loads the tile plus a
// halo (HX columns, HY rows on each side) into shared memory with one TMA
// tensor copy, then runs K sub-steps entirely in shared memory.  Its warps have
// two roles that meet on two named barriers per sub-step:
//   cone warps (2)   hold up to 192 of the tile's cones in registers; before
//                    the first barrier each samples C^{n+j} at its cones (the
//                    multilinear gradient from 12 patch nodes), after it the
//                    rest of step n+j (Philox noise, blend, advance, stop tests),
//                    which reads no field, runs while the field warps sweep;
//   field warps (8)  before the first barrier step any further cones of the
//                    bin (state in global memory) on C^{n+j}; after it each
//                    sweeps a band of full-width rows in place to C^{n+j+1},
//                    keeping the rows above/at/below in registers (x neighbours
//                    by warp shuffle) and adding the point sources of each row.
// The cone work thus overlaps the sweep instead of holding every warp at a
// CTA barrier (measured on the 2048^2 workload: 35.9 -> 30.8 us per 8-step
// launch; one cone warp, or three or four, were slower: one is starved of issue
// slots by the sweeping warps, more lower the register budget of the sweep;
// letting the cone warps also step the bin's further cones cost 2.5 us per
// launch on the uniform workload and saved 2% on the clustered one).
// After K sub-steps the interior is stored.  The valid region shrinks by one
// node per sub-step; cones move at most step_len per step and read a 4-node
// footprint, so the halo is H = K + 1 + ceil((K-1) step_len / h) (the x halo
// rounded up to 4 nodes for 16-byte TMA coordinates).  Each launch re-bins its
// cones for the next one as they finish: per-tile bins filled through atomic
// counters.  A bin holds every cone of its tile whenever the bins fit the
// workspace budget (then no cone ever spills, however the cones cluster); the
// first 192 ids of a bin ride in the cone warps' registers for the whole launch,
// the rest are stepped by the field warps from global memory.  Only on grids too large for such bins does a
// bin hold 512 ids, cones of a full bin going to a spill list that every tile
// scans.  Each tile clears its own count once read, the last tile past its
// prologue clears the spill count.  No separate binning launch between fused
// launches.
// Crowded tiles: a launch may carry helper blocks at the start of its grid.
// Each sweeps a crowded tile's field and steps one slice of kHelpCap of its
// cones (a tile's own block steps the first slice and what its helpers do not
// cover), so a tile holding thousands of cones no longer makes the launch wait
// for one block.  The helper count comes from the crowding the previous run
// reported (a count kept as cones are re-binned, read back without blocking).

//
// Model: cue field on an Eulerian grid (Sec. 5.2) with sources of their own
// rates (Sec. 4.3); cone steering by vector addition (Sec. 3.5, Eq. 6-7) with
// stateless counter-based noise (Sec. 5.1) and Box-Muller (Sec. 3.2); stop
// tests on the bounds (Sec. 3.4) and squared source distance (Sec. 3.3).
// The paper's own GPU design sorts particles into a uniform grid by cell hash
// (Sec. 3.5, calculateHash / identifyCellStart); the binning here is the same
// idea applied to cones and field tiles.
#include <cuda.h>

#include <cmath>

#include "cue_internal.h"
#include "cue_tile.cuh"

namespace cue {
namespace {

using namespace tile;

constexpr int kMaxTileSrc = 256;      // sources inside one tile's loaded region
constexpr int kMaxFusedSources = 1 << 16;   // sources in total on this path (each tile scans them all)
constexpr int kFusedMinTX = 128;      // smallest interior tile the path accepts
constexpr int kFusedMinTY = 32;

struct FusedArgs {
    FieldDesc f;
    ConeDesc c;
    FusedGeom g;
    float *Cout;
    int K;
    uint32_t step0;
    int cones_on;
    int n_axons;
    float *pos, *dir;
    uint8_t *active;
    // this launch's bins: count (each tile clears its own after reading it),
    // ids, and the spill list of cones whose bin was full
    int *cnt_cur;
    const int *bins_cur;
    const int2 *spill_cur;
    int *spill_cnt_cur;
    // the next launch's bins, filled as the cones finish (null: no re-binning)
    int *cnt_next;
    int *bins_next;
    int2 *spill_next;
    int *spill_cnt_next;
    int *done;                                 // CTAs past their prologue: the last clears spill_cnt_cur
    int n_help;                                // helper CTAs at the start of the grid (0: none)
    int round;                                 // bin round this launch reads
    int n_tiles;
    int *need;                                 // [0] the run's largest per-launch helper need; [1 + round]
                                               // the need of the bins filled for that round
    int bin_cap;                               // ids per tile bin (this launch's and the next's)
    const int32_t *src_cell;
    const float *src_emit;
    int n_src;
    const float *src_xyz;
    unsigned *status;
    unsigned long long *counter;
};

constexpr int kHelpCap = 192;          // cones per CTA when a crowded tile's cones are shared out (its register slots)
constexpr int kHelpMaxTiles = 2048;    // grids with more tiles run without helpers
constexpr int kMaxHelpers = 128;
constexpr int kConeWarps = 2;          // warps that step the cones, after the 8 field warps
constexpr int kConeSlots = 3;          // cones held in registers per lane of a cone warp
constexpr int kRegCones = kConeSlots * 32 * kConeWarps;   // the first kRegCones ids of a bin ride in registers
constexpr int kFusedThreads = kThreads + 32 * kConeWarps;
static_assert(kHelpCap <= kRegCones, "a helper's cones ride in the cone warps' registers");

// The helper need of the bins this launch reads is complete (the launch that filled
// them has finished): fold it into the run's maximum and clear its slot for the
// launch after next.  Called once per launch, by the last CTA past its prologue.
__device__ __forceinline__ void fold_need(const FusedArgs &A)
{
    int *slot = &A.need[1 + A.round];
    if (*slot > A.need[0]) A.need[0] = *slot;
    *slot = 0;
}

// Named barriers between the field warps and the cone warps (every warp arrives
// converged, from its own role's loop).
__device__ __forceinline__ void role_sync(int id)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kFusedThreads) : "memory");
}

__device__ __forceinline__ int tile_of(const FieldDesc &f, const FusedGeom &g, float px, float py)
{
    int ix = clampi((int)floorf(px * f.inv_h), 0, f.nx - 1);
    int iy = clampi((int)floorf(py * f.inv_h), 0, f.ny - 1);
    return (iy / g.TY) * g.ntx + ix / g.TX;
}

// HELP: the launch may carry helper blocks (n_help > 0); without it the kernel is the
// plain one-tile-per-block form.
template <bool HELP>
__global__ void __launch_bounds__(kFusedThreads, 2) fused2d_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                   const FusedArgs A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const FusedGeom &g = A.g;
    const FieldDesc &f = A.f;
    // layout: mbarrier at 0; the TMA tile at 128 (128-byte aligned); then the lists
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    float *S = reinterpret_cast<float *>(smem_raw + 128);
    float4 *S4 = reinterpret_cast<float4 *>(smem_raw + 128);
    int *row_start = reinterpret_cast<int *>(S + kRows * kW);    // R + 1
    int *row_fill = row_start + (kRows + 1);                      // R
    int *t_col = row_fill + kRows;                                // kMaxTileSrc each:
    int *t_row = t_col + kMaxTileSrc;
    float *t_e = reinterpret_cast<float *>(t_row + kMaxTileSrc);
    float *t_xy = t_e + kMaxTileSrc;                            // [2][kMaxTileSrc] tile sources

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool cone_warp = warp >= kWarps;        // warps 0-7 sweep the field, warps 8-9 step the cones
    const int n = A.n_axons;
    // Work item of this CTA.  Without helpers (n_help == 0) CTA b is tile b.  With
    // helpers the first n_help CTAs are helpers: each takes a slice of kHelpCap cones
    // of a crowded tile (a tile whose bin holds more than kHelpCap cones), sweeps that
    // tile's field in its own shared memory and steps only its slice; the other CTAs
    // are the tiles, in order, each stepping its first kHelpCap cones plus whatever
    // its helpers do not cover.  Helpers past the work exit.
    const bool stop_on = A.cones_on && A.c.stop_r2 >= 0.0f && A.n_src > 0;
    const bool helper = HELP && (int)blockIdx.x < A.n_help;
    int t = HELP ? (helper ? -1 : (int)blockIdx.x - A.n_help) : (int)blockIdx.x;   // a helper's tile comes from the plan
    __shared__ int s_item[4];                      // helper: tile, slice; tile CTA: helpers it has

    // Point sources inside the loaded region of tile (ox, oy), grouped by tile row.
    auto build_sources = [&](int ox, int oy, bool report) {
        for (int r = tid; r < kRows; r += kFusedThreads) row_fill[r] = 0;
        __syncthreads();
        for (int s = tid; s < A.n_src && tid < kThreads; s += kThreads) {
            int cell = A.src_cell[s];
            if (cell >= 0 && cell < f.nx * f.ny) {
                int gx = cell % f.nx, gy = cell / f.nx;
                if (gx >= ox && gx < ox + kW && gy >= oy && gy < oy + kRows) atomicAdd(&row_fill[gy - oy], 1);
            } else if (report) {
                flag_status(A.status, kStatusBounds);      // skipped, reported once per launch
            }
        }
        __syncthreads();
        if (warp == 0) {       // exclusive scan of the per-row counts
            int carry = 0;
            for (int base = 0; base < kRows; base += 32) {
                int r = base + lane;
                int v = r < kRows ? row_fill[r] : 0;
                int x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(kFull, x, o);
                    if (lane >= o) x += y;
                }
                if (r < kRows) row_start[r] = carry + x - v;
                carry += __shfl_sync(kFull, x, 31);
            }
            if (lane == 0) row_start[kRows] = carry;
        }
        __syncthreads();
        for (int r = tid; r < kRows; r += kFusedThreads) row_fill[r] = 0;
        __syncthreads();
        for (int s = tid; s < A.n_src && tid < kThreads; s += kThreads) {
            int cell = A.src_cell[s];
            if (cell >= 0 && cell < f.nx * f.ny) {
                int gx = cell % f.nx, gy = cell / f.nx;
                if (gx >= ox && gx < ox + kW && gy >= oy && gy < oy + kRows) {
                    int r = gy - oy;
                    int slot = row_start[r] + atomicAdd(&row_fill[r], 1);
                    t_col[slot] = gx - ox;
                    t_row[slot] = r;
                    t_e[slot] = A.src_emit[s];
                    t_xy[slot] = (float)gx * f.h;
                    t_xy[kMaxTileSrc + slot] = (float)gy * f.h;
                }
            }
        }
    };

    // Programmatic dependent launch: the next launch's CTAs may be scheduled as this
    // launch's CTAs finish.  Up to griddepcontrol.wait a tile CTA reads only inputs that
    // no kernel writes (the point sources), so that part of its prologue overlaps the
    // previous launch's last tiles; the wait (a no-op in a launch without the
    // attribute) returns once the previous launch has completed and its writes are
    // visible.  A helper learns its tile from the bins, after the wait.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) mbar_init(bar, 1);
    // a tile CTA's load coordinates, ready before the wait (the copy is the first thing after it)
    const int tox = helper ? 0 : t % g.ntx * g.TX - g.HX, toy = helper ? 0 : t / g.ntx * g.TY - g.HY;
    if (!helper) build_sources(tox, toy, t == 0);

    // from here on: what earlier launches wrote (the field, the cone bins and state)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    auto issue_tile = [&](int x, int y) {
        if (tid == 0) {
            mbar_expect_tx(bar, (unsigned)(kRows * kW * sizeof(float)));
            tma_load_2d(S, &tmap, bar, x, y);
        }
    };
    if (!helper) issue_tile(tox, toy);              // a tile CTA's copy goes out first

    // The helper plan: every tile's helper need (its cones past kHelpCap, kHelpCap per
    // helper), scanned over the tiles in the order of the tile index.  Only helpers and
    // crowded tiles (of a launch with helpers) compute it.
    const int nb_own = (HELP && A.cones_on && !helper) ? min(A.cnt_cur[t], A.bin_cap) : 0;
    const int need_own = nb_own > kHelpCap ? (nb_own - 1) / kHelpCap : 0;
    if (HELP && A.cones_on && (helper || need_own > 0) && A.n_tiles <= kHelpMaxTiles) {
        __shared__ int s_wsum[kFusedThreads / 32];
        const int per = (A.n_tiles + kFusedThreads - 1) / kFusedThreads;
        const int t_lo = min(tid * per, A.n_tiles), t_hi = min(t_lo + per, A.n_tiles);
        auto need_of_tile = [&](int tt) {
            const int nb = min(A.cnt_cur[tt], A.bin_cap);
            return nb > kHelpCap ? (nb - 1) / kHelpCap : 0;
        };
        int mine = 0;
        for (int tt = t_lo; tt < t_hi; ++tt) mine += need_of_tile(tt);
        int x = mine;                                   // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        if (tid == 0) {
            s_item[0] = -1;
            s_item[2] = 0;
        }
        __syncthreads();
        int before = x - mine, total = 0;
        for (int w = 0; w < kFusedThreads / 32; ++w) {
            if (w < warp) before += s_wsum[w];
            total += s_wsum[w];
        }
        const int used = min(total, A.n_help);
        int pre = before;
        for (int tt = t_lo; tt < t_hi; ++tt) {
            const int nd = need_of_tile(tt);
            if (helper) {
                const int h = (int)blockIdx.x;
                if (h >= pre && h < pre + nd && h < used) {
                    s_item[0] = tt;
                    s_item[1] = h - pre + 1;               // slice 1.. of the tile's bin
                }
            } else if (tt == t) {
                s_item[2] = min(max(used - pre, 0), nd);   // helpers this tile has
            }
            pre += nd;
        }
        __syncthreads();
        if (helper) t = s_item[0];
    }
    if (helper && t < 0) {                          // no work: count in and leave
        if (tid == 0 && atomicAdd(A.done, 1) == (int)gridDim.x - 1) {
            for (int tt = 0; tt < A.n_tiles; ++tt) A.cnt_cur[tt] = 0;
            fold_need(A);
            *A.spill_cnt_cur = 0;
            *A.done = 0;
        }
        return;
    }
    const int tx = t % g.ntx, ty = t / g.ntx;
    const int ox = tx * g.TX - g.HX, oy = ty * g.TY - g.HY;
    if (helper) {
        issue_tile(ox, oy);
        build_sources(ox, oy, false);
    }

    // this CTA's cones into registers (overlaps the TMA load): its list is one or two
    // ranges of the tile's bin -- a helper: slice s, [s kHelpCap, (s + 1) kHelpCap);
    // a tile with helpers: [0, kHelpCap) and what follows its helpers' slices
    __shared__ int s_nspill;
    if (tid == 0) s_nspill = A.cones_on ? *A.spill_cnt_cur : 0;
    const int n_bin_all = A.cones_on ? min(A.cnt_cur[t], A.bin_cap) : 0;
    int b1 = 0, L1 = n_bin_all, b2 = 0, L2 = 0;
    if (HELP && A.cones_on) {
        if (helper) {
            b1 = s_item[1] * kHelpCap;
            L1 = min(kHelpCap, n_bin_all - b1);
        } else if (n_bin_all > kHelpCap) {
            L1 = kHelpCap;
            b2 = kHelpCap * (1 + s_item[2]);
            L2 = max(n_bin_all - b2, 0);
        }
    }
    const int n_bin = L1 + L2;
    const int *bin_base = A.bins_cur + (size_t)t * A.bin_cap;
    auto bin_at = [&](int i) { return HELP ? bin_base[i < L1 ? b1 + i : b2 + (i - L1)] : bin_base[i]; };
    // the cone warps' slots: list entry (32 q + lane) kConeWarps + w in slot q of lane
    // `lane` of cone warp w, so a CTA's cones are shared out evenly (the rest of the
    // list, if any, is stepped by the field warps from global memory)
    int ca[kConeSlots];
    bool cl[kConeSlots];
    float cp[kConeSlots][2], cdir[kConeSlots][2];
#pragma unroll
    for (int q = 0; q < kConeSlots; ++q) {
        const int i = (32 * q + lane) * kConeWarps + (warp - kWarps);
        ca[q] = cone_warp && i < n_bin ? bin_at(i) : -1;
        cl[q] = ca[q] >= 0;
        if (cl[q]) {
            cl[q] = A.active[ca[q]] != 0;
            cp[q][0] = A.pos[ca[q]];
            cp[q][1] = A.pos[n + ca[q]];
            cdir[q][0] = A.dir[ca[q]];
            cdir[q][1] = A.dir[n + ca[q]];
        }
    }
    __syncthreads();
    const int n_spill = s_nspill;
    if (A.cones_on && tid == 0) {
        // every thread has read this tile's count: clear it for the launch after next
        // (with helpers every CTA read every count: the last CTA past this point clears
        // them all); the last CTA past this point clears the spill count
        if (!HELP) A.cnt_cur[t] = 0;
        if (atomicAdd(A.done, 1) == (int)gridDim.x - 1) {
            if (HELP)
                for (int tt = 0; tt < A.n_tiles; ++tt) A.cnt_cur[tt] = 0;
            fold_need(A);
            *A.spill_cnt_cur = 0;
            *A.done = 0;
        }
    }

    // wait for the tile: one thread polls (bounded), the rest wait at the barrier
    bool ok = true;
    if (tid == 0) ok = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            flag_status(A.status, kStatusTimeout);
            mbar_wait_bounded(bar, 0);      // let an in-flight copy land before the CTA exits
        }
        return;
    }
    mbar_wait_bounded(bar, 0);              // completed phase: returns at once, acquires the tile

    const int r0 = cone_warp ? 0 : warp * kBand;
    const int colA = 4 * lane, colB = 128 + 4 * lane;
    const int gxA = ox + colA, gxB = ox + colB;
    const float2 alpha2 = make_float2(f.alpha, f.alpha), beta2 = make_float2(f.beta, f.beta);
    const BandSources bsrc{t_col, t_row, t_e, row_start[r0], row_start[r0 + kBand]};
    // source-stop list: this tile's sources when the halo covers the stop radius, else all
    const float *stop_xy = g.local_stop ? t_xy : A.src_xyz;
    const int stop_stride = g.local_stop ? kMaxTileSrc : A.n_src;
    const int n_stop = stop_on ? (g.local_stop ? row_start[kRows] : A.n_src) : 0;
    // walls: x walls by per-lane flags; y walls by a ghost row inside the loaded rows
    const LaneWalls lw = lane_walls(gxA, gxB, f.nx);      // nx % 4 == 0 on this path: walls on group edges
    const BandMap no_map{};
    const int gt = (oy <= -1) ? -oy - 1 : -1;                       // tile row of global y = -1
    const int gb = (oy + kRows - 1 >= f.ny) ? f.ny - oy : -1;       // tile row of global y = ny
    const bool wall = gt >= 0 || gb >= 0;
    if (wall) {       // ghost rows take the edge rows before the first sub-step
        if (gt >= 0)
            for (int c = tid; c < kW; c += kThreads) S[gt * kW + c] = S[(gt + 1) * kW + c];
        if (gb >= 0 && gb < kRows)
            for (int c = tid; c < kW; c += kThreads) S[gb * kW + c] = S[(gb - 1) * kW + c];
        __syncthreads();
    }

    auto ld = [&](int i, int j, int) {
        int lx = i - ox, ly = j - oy;
        if ((unsigned)lx >= (unsigned)kW || (unsigned)ly >= (unsigned)kRows) {
            flag_status(A.status, kStatusBounds);
            lx = min(max(lx, 0), kW - 1);
            ly = min(max(ly, 0), kRows - 1);
        }
        return S[ly * kW + lx];
    };

    auto ld_fast = [&](int i, int j, int) { return S[(j - oy) * kW + (i - ox)]; };
    // the field-dependent part of a cone step: the multilinear gradient at p from
    // the 12 patch nodes in shared memory (the plain kernel's arithmetic)
    auto grad_at = [&](const float *p, float *gr) {
        int lo[2];
        float fr[2], v[kPatch2];
        cell_of<2>(f, p, lo, fr);
        const bool inside = max(lo[0] - 1, 0) - ox >= 0 && min(lo[0] + 2, f.nx - 1) - ox < kW &&
                            max(lo[1] - 1, 0) - oy >= 0 && min(lo[1] + 2, f.ny - 1) - oy < kRows;
        if (inside) gather2(f, lo, ld_fast, v);
        else gather2(f, lo, ld, v);
        grad2(A.c, v, fr, gr);
    };
    // one whole cone step on the shared-memory field
    auto step_cone = [&](uint32_t a, uint32_t stp, float *p, float *d) {
        float gr[2], xi[2];
        grad_at(p, gr);
        cone_noise<2>(A.c.key0, A.c.key1, a, stp, xi);
        return cone_finish_xi<2>(A.c, gr, xi, p, d, stop_xy, stop_stride, n_stop);
    };
    auto rebin = [&](int a, float px, float py) {
        const int tile = tile_of(f, g, px, py);
        const int slot = atomicAdd(&A.cnt_next[tile], 1);
        // a bin passing a multiple of kHelpCap cones needs one more helper: the run's
        // total, from which the host sizes the next run's helpers
        if (slot >= kHelpCap && slot % kHelpCap == 0) atomicAdd(&A.need[1 + (A.round ^ 1)], 1);
        if (slot < A.bin_cap) {
            A.bins_next[(size_t)tile * A.bin_cap + slot] = a;
        } else {
            const int k = atomicAdd(A.spill_cnt_next, 1);
            A.spill_next[k] = make_int2(a, tile);
        }
    };

    if (cone_warp) {
        // ---- the cone warps.  Sub-step j: the slot cones sample C^{n+j} (their
        // gradients), the first barrier lets the field warps overwrite it, and the
        // rest of step n+j (noise, steering, advance, stop tests), which reads no
        // field, runs while the field warps sweep; the second barrier ends the sub-step.
        bool stopped[kConeSlots];
#pragma unroll
        for (int q = 0; q < kConeSlots; ++q) stopped[q] = false;
        for (int j = 0; j < A.K; ++j) {
            const uint32_t step = A.step0 + j;
            float cg[kConeSlots][2];
#pragma unroll
            for (int q = 0; q < kConeSlots; ++q) {
                cg[q][0] = cg[q][1] = 0.f;
                if (cl[q]) grad_at(cp[q], cg[q]);
            }
            role_sync(1);
#pragma unroll
            for (int q = 0; q < kConeSlots; ++q) {
                count_active(A.counter, cl[q]);
                if (cl[q]) {
                    float xi[2];
                    cone_noise<2>(A.c.key0, A.c.key1, (uint32_t)ca[q], step, xi);
                    if (!cone_finish_xi<2>(A.c, cg[q], xi, cp[q], cdir[q], stop_xy, stop_stride, n_stop)) {
                        cl[q] = false;
                        stopped[q] = true;
                    }
                }
            }
            role_sync(2);
        }
        // the slot cones back to global memory, binned for the next launch
#pragma unroll
        for (int q = 0; q < kConeSlots; ++q) {
            const int a = ca[q];
            if (a < 0) continue;
            A.pos[a] = cp[q][0];
            A.pos[n + a] = cp[q][1];
            A.dir[a] = cdir[q][0];
            A.dir[n + a] = cdir[q][1];
            if (stopped[q]) A.active[a] = 0;
            if (A.cnt_next && cl[q]) rebin(a, cp[q][0], cp[q][1]);
        }
        return;
    }

    // ---- the field warps
    for (int j = 0; j < A.K; ++j) {
        const uint32_t step = A.step0 + j;
        // cones of the bin beyond the cone warps' slots, then the spilled cones of this
        // tile: whole steps on C^{n+j}, state read from and written back to global memory
        // (warp-uniform trip counts: count_active is a warp-collective ballot);
        // software-pipelined: the next round's cone state (and the ids two rounds ahead)
        // are loaded while this round's cone steps, so a crowded tile is bound by its
        // arithmetic rather than by chains of dependent loads
        if (n_bin > kRegCones) {
            auto id_at = [&](int i) { return i < n_bin ? bin_at(i) : -1; };
            int a_nn = id_at(kRegCones + kThreads + tid);
            int a_n = id_at(kRegCones + tid);
            bool live_n = a_n >= 0 && A.active[a_n] != 0;
            float p_n[2] = {0.f, 0.f}, d_n[2] = {0.f, 0.f};
            if (live_n) {
                p_n[0] = A.pos[a_n];
                p_n[1] = A.pos[n + a_n];
                d_n[0] = A.dir[a_n];
                d_n[1] = A.dir[n + a_n];
            }
            for (int base = kRegCones; base < n_bin; base += kThreads) {
                const int a = a_n;
                const bool live = live_n;
                float p[2] = {p_n[0], p_n[1]}, d[2] = {d_n[0], d_n[1]};
                a_n = a_nn;                                   // next round: state in flight now
                a_nn = id_at(base + 2 * kThreads + tid);        // the round after next
                live_n = a_n >= 0 && A.active[a_n] != 0;
                if (live_n) {
                    p_n[0] = A.pos[a_n];
                    p_n[1] = A.pos[n + a_n];
                    d_n[0] = A.dir[a_n];
                    d_n[1] = A.dir[n + a_n];
                }
                count_active(A.counter, live);             // warp-uniform trip count
                if (live) {
                    bool alive = step_cone((uint32_t)a, step, p, d);
                    A.pos[a] = p[0];
                    A.pos[n + a] = p[1];
                    A.dir[a] = d[0];
                    A.dir[n + a] = d[1];
                    if (!alive) A.active[a] = 0;
                }
            }
        }
        for (int base = 0; base < n_spill; base += kThreads) {   // spilled cones of this tile
            const int i = base + tid;
            const int2 e = i < n_spill ? A.spill_cur[i] : make_int2(-1, -1);
            const int a = e.y == t ? e.x : -1;
            bool live = a >= 0 && A.active[a];
            count_active(A.counter, live);
            if (live) {
                float p[2] = {A.pos[a], A.pos[n + a]};
                float d[2] = {A.dir[a], A.dir[n + a]};
                bool alive = step_cone((uint32_t)a, step, p, d);
                A.pos[a] = p[0];
                A.pos[n + a] = p[1];
                A.dir[a] = d[0];
                A.dir[n + a] = d[1];
                if (!alive) A.active[a] = 0;
            }
        }
        // rows just outside this warp's band, read before anyone overwrites them
        const Row above = ld_row(S4, r0 > 0 ? r0 - 1 : r0, lane);
        const Row below = ld_row(S4, r0 + kBand < kRows ? r0 + kBand : r0 + kBand - 1, lane);
        role_sync(1);
        // ---- in-place sweep of the band to C^{n+j+1}
        if (wall) sweep_band<true, false, false>(S4, lane, r0, above, below, lw, alpha2, beta2, bsrc, oy, f.ny, no_map);
        else sweep_band<false, false, false>(S4, lane, r0, above, below, lw, alpha2, beta2, bsrc, oy, f.ny, no_map);
        role_sync(2);
    }

    // ---- the other cones back to their bins for the next launch
    if (A.cnt_next) {
        for (int i = kRegCones + tid; i < n_bin; i += kThreads) {
            const int a = bin_at(i);
            if (A.active[a]) rebin(a, A.pos[a], A.pos[n + a]);
        }
        for (int i = tid; i < n_spill; i += kThreads) {
            const int2 e = A.spill_cur[i];
            if (e.y == t && A.active[e.x]) rebin(e.x, A.pos[e.x], A.pos[n + e.x]);
        }
    }

    // ---- store the interior (a helper's copy of the tile is not stored)
    if (helper) return;
    bool bad = false;
    for (int r = g.HY + warp; r < g.HY + g.TY; r += kWarps) {
        const int gy = oy + r;
        if (gy >= f.ny) break;
        float4 *out = reinterpret_cast<float4 *>(A.Cout + (size_t)gy * f.nx);
        if (colA >= g.HX && colA < g.HX + g.TX && gxA < f.nx) {
            float4 v = S4[r * (kW / 4) + lane];
            bad |= !(fabsf(v.x) <= 3.4e38f && fabsf(v.y) <= 3.4e38f && fabsf(v.z) <= 3.4e38f &&
                     fabsf(v.w) <= 3.4e38f);
            out[gxA >> 2] = v;
        }
        if (colB >= g.HX && colB < g.HX + g.TX && gxB < f.nx) {
            float4 v = S4[r * (kW / 4) + 32 + lane];
            bad |= !(fabsf(v.x) <= 3.4e38f && fabsf(v.y) <= 3.4e38f && fabsf(v.z) <= 3.4e38f &&
                     fabsf(v.w) <= 3.4e38f);
            out[gxB >> 2] = v;
        }
    }
    if (__any_sync(kFull, bad) && lane == 0) flag_status(A.status, kStatusNonFinite);
}

// ---------------------------------------------------------------- binning
// Start of a run: every active cone into its tile's bin (or the spill list).
__global__ void bin_count_kernel(FieldDesc f, FusedGeom g, int n, const float *__restrict__ pos,
                                 const uint8_t *__restrict__ active, int *count, int *bins, int bin_cap,
                                 int2 *spill, int *spill_cnt)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n || !active[a]) return;
    const int tile = tile_of(f, g, pos[a], pos[n + a]);
    const int slot = atomicAdd(&count[tile], 1);
    if (slot < bin_cap) {
        bins[(size_t)tile * bin_cap + slot] = a;
    } else {
        const int k = atomicAdd(spill_cnt, 1);
        spill[k] = make_int2(a, tile);
    }
}

// ---------------------------------------------------------------- host side
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

int device_sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 152;
}

size_t fused_smem_bytes(int R)
{
    return 128 + (size_t)R * kW * sizeof(float) + sizeof(int) * (2 * R + 1) + sizeof(int) * 2 * kMaxTileSrc +
           sizeof(float) * 3 * kMaxTileSrc;
}

// Tile geometry for temporal depth K; returns false if the fused path cannot run.
bool choose_geometry(const FieldDesc &f, float step_len, float stop_r2, bool cones, int K, int sms, FusedGeom &g)
{
    if (f.dim != 2 || K < 1 || K > kMaxTemporalDepth) return false;
    const double tol = 1.0 + 1e-5;
    double drift = cones ? std::ceil((K - 1) * (double)step_len / (double)f.h * tol) : 0.0;
    int H = cones ? (int)(K + 1 + drift) : K;
    // a cone stays within K step_len of its tile; sources within the stop radius of it
    // are then inside the loaded region when H >= ceil((K step_len + r) / h) + 1
    int local_stop = 1;
    if (cones && stop_r2 >= 0.0f) {
        double r = std::sqrt((double)stop_r2);
        int need = (int)std::ceil((K * (double)step_len + r) / (double)f.h * tol) + 1;
        local_stop = need <= H ? 1 : 0;
    }
    int HX = (H + 3) & ~3;
    const int R = kRows, cps = 2;
    int TY = R - 2 * H;
    int TX = kW - 2 * HX;
    // tiles smaller than this are mostly halo (and the workspace's bins are sized for
    // no more tiles than these interiors give): every depth up to 16 with step_len <= h
    if (TX < kFusedMinTX || TY < kFusedMinTY) return false;
    g.W = kW;
    g.R = R;
    g.HX = HX;
    g.HY = H;
    g.TX = TX;
    g.TY = TY;
    g.ntx = (f.nx + TX - 1) / TX;
    g.nty = (f.ny + TY - 1) / TY;
    g.K = K;
    g.ctas_per_sm = cps;
    g.local_stop = local_stop;
    (void)sms;
    bool found = true;
    return found;
}

}  // namespace

bool fused_geometry(const FieldDesc &f, float step_len, float stop_r2, bool cones, int K, FusedGeom &g)
{
    return choose_geometry(f, step_len, stop_r2, cones, K, device_sm_count(), g);
}

bool encode_field_map_available() { return encode_fn() != nullptr; }

bool encode_field_map(void *map128, float *base, int nx, int ny, int pitch)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)kW, (cuuint32_t)kRows};
    cuuint32_t estr[2] = {1, 1};
    return fn(reinterpret_cast<CUtensorMap *>(map128), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Upper bound on the tile count of any accepted geometry (interior at least
// kFusedMinTX x kFusedMinTY), used to size the binning workspace independently
// of the temporal depth.
int fused_tile_count(const cue_params &p)
{
    if (p.dim != 2) return 0;
    long long n = (long long)((p.nx + kFusedMinTX - 1) / kFusedMinTX) * ((p.ny + kFusedMinTY - 1) / kFusedMinTY);
    return n > (1 << 22) ? 0 : (int)n;
}

static int default_depth(const Sim &s) { return s.temporal_depth > 0 ? s.temporal_depth : 8; }

// Whether no tile's loaded region (kW x R nodes from (tx TX - HX, ty TY - HY)) holds
// more than kMaxTileSrc point sources, the size of a tile's source list in shared
// memory.  Up to kMaxTileSrc sources in total always fit; past that the source
// cells are copied to the host once per handle (a synchronous copy) and counted
// per region, once per geometry.  Inside a stream capture no copy is made and the
// path is refused.
static bool fused_sources_fit(const Sim &s, const FusedGeom &g)
{
    if (s.n_src <= kMaxTileSrc) return true;
    if (s.src_fit_K == g.K) return s.src_fit_ok;
    if (s.src_cells_host.empty()) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s.stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return false;
        std::vector<int32_t> cells((size_t)s.n_src);
        if (cudaStreamSynchronize(s.stream) != cudaSuccess ||
            cudaMemcpy(cells.data(), s.src_cell, sizeof(int32_t) * cells.size(), cudaMemcpyDeviceToHost) !=
                cudaSuccess)
            return false;
        s.src_cells_host.swap(cells);
    }
    std::vector<int> count((size_t)g.ntx * g.nty, 0);
    bool ok = true;
    for (int32_t cell : s.src_cells_host) {
        if (cell < 0 || cell >= s.fd.nx * s.fd.ny) continue;     // skipped (and reported) by the kernel
        const int gx = cell % s.fd.nx, gy = cell / s.fd.nx;
        // tiles whose loaded region holds (gx, gy): tx TX - HX <= gx < tx TX - HX + kW
        const int tx_lo = std::max(0, (gx + g.HX - kW + g.TX) / g.TX), tx_hi = std::min(g.ntx - 1, (gx + g.HX) / g.TX);
        const int ty_lo = std::max(0, (gy + g.HY - g.R + g.TY) / g.TY), ty_hi = std::min(g.nty - 1, (gy + g.HY) / g.TY);
        for (int ty = ty_lo; ty <= ty_hi && ok; ++ty)
            for (int tx = tx_lo; tx <= tx_hi && ok; ++tx) {
                const int ox = tx * g.TX - g.HX, oy = ty * g.TY - g.HY;
                if (gx < ox || gx >= ox + kW || gy < oy || gy >= oy + g.R) continue;
                if (++count[(size_t)ty * g.ntx + tx] > kMaxTileSrc) ok = false;
            }
    }
    s.src_fit_K = g.K;
    s.src_fit_ok = ok;
    return ok;
}

bool fused_supported(const Sim &s)
{
    if (s.fd.dim != 2 || !s.vec4 || s.src_map || s.n_src > kMaxFusedSources || s.cd.steer != 0) return false;
    if (!encode_fn()) return false;
    FusedGeom g;
    if (!choose_geometry(s.fd, s.cd.step_len, s.cd.stop_r2, s.n_axons > 0, default_depth(s), device_sm_count(), g))
        return false;
    long long tiles = (long long)g.ntx * g.nty;
    if (tiles > s.wl.n_tiles) return false;             // the workspace's bins are sized by fused_tile_count
    if (!fused_sources_fit(s, g)) return false;
    return true;
}

static bool make_maps(Sim &s)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    for (int b = 0; b < 2; ++b) {
        cuuint64_t dims[2] = {(cuuint64_t)s.fd.nx, (cuuint64_t)s.fd.ny};
        cuuint64_t strides[1] = {(cuuint64_t)s.fd.nx * sizeof(float)};
        cuuint32_t box[2] = {(cuuint32_t)kW, (cuuint32_t)s.geom.R};
        cuuint32_t estr[2] = {1, 1};
        CUresult r = fn(reinterpret_cast<CUtensorMap *>(s.tmap[b]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, s.field[b],
                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

static int prepare(Sim &s)
{
    const int K = default_depth(s);
    if (s.geom_ready && s.geom.K == K) return CUE_OK;
    FusedGeom g;
    if (!choose_geometry(s.fd, s.cd.step_len, s.cd.stop_r2, s.n_axons > 0, K, device_sm_count(), g))
        return CUE_ERR_ARG;
    s.geom = g;
    if (!make_maps(s)) return CUE_ERR_CUDA;
    size_t smem = fused_smem_bytes(g.R);
    if (cudaFuncSetAttribute(fused2d_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(fused2d_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return CUE_ERR_CUDA;
    s.geom_ready = true;
    return CUE_OK;
}

// Bin every active cone for the current round (start of a run); both rounds'
// counts and spill counts start at zero.
static cudaError_t launch_bin_count(Sim &s)
{
    const int n_tiles = s.geom.ntx * s.geom.nty;
    const int r = (int)(s.bin_round & 1);
    cudaError_t e = cudaMemsetAsync(s.bin_count(), 0, sizeof(int) * 2 * s.wl.n_tiles, s.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.bin_ctl(), 0, 256, s.stream);
    if (e != cudaSuccess) return e;
    bin_count_kernel<<<(s.n_axons + 255) / 256, 256, 0, s.stream>>>(
        s.fd, s.geom, s.n_axons, s.pos, s.active, s.bin_count() + r * s.wl.n_tiles,
        s.bin_list() + (size_t)r * s.wl.n_tiles * s.wl.bin_cap, s.wl.bin_cap, s.spill() + (size_t)r * s.n_axons,
        s.bin_ctl() + r);
    (void)n_tiles;
    s.launches++;
    return cudaGetLastError();
}

// One launch of k <= K fused steps (cones on or off) from s.cur into s.cur^1.
// With cones: the kernel reads the current round's bins and fills the next's.
static cudaError_t launch_fused(Sim &s, int k, bool cones, int n_help = 0)
{
    const FusedGeom &g = s.geom;
    const int n_tiles = g.ntx * g.nty;
    const bool with_cones = cones && s.n_axons > 0;
    const int r = (int)(s.bin_round & 1), rn = r ^ 1;
    FusedArgs A;
    A.f = s.fd;
    A.c = s.cd;
    A.g = g;
    A.Cout = s.field[s.cur ^ 1];
    A.K = k;
    A.step0 = (uint32_t)s.field_step;
    A.cones_on = with_cones ? 1 : 0;
    A.n_axons = s.n_axons;
    A.pos = s.pos;
    A.dir = s.dir;
    A.active = s.active;
    A.cnt_cur = s.bin_count() + r * s.wl.n_tiles;
    A.bins_cur = s.bin_list() + (size_t)r * s.wl.n_tiles * s.wl.bin_cap;
    A.spill_cur = s.spill() + (size_t)r * s.n_axons;
    A.spill_cnt_cur = s.bin_ctl() + r;
    A.cnt_next = with_cones ? s.bin_count() + rn * s.wl.n_tiles : nullptr;
    A.bins_next = s.bin_list() + (size_t)rn * s.wl.n_tiles * s.wl.bin_cap;
    A.spill_next = s.spill() + (size_t)rn * s.n_axons;
    A.spill_cnt_next = s.bin_ctl() + rn;
    A.done = s.bin_ctl() + 2;
    A.need = s.bin_ctl() + 3;
    A.round = r;
    A.n_tiles = n_tiles;
    A.n_help = with_cones ? n_help : 0;
    A.bin_cap = s.wl.bin_cap;
    A.src_cell = s.src_cell;
    A.src_emit = s.src_emit;
    A.n_src = s.n_src;
    A.src_xyz = s.src_xyz();
    A.status = s.status();
    A.counter = s.cone_counter();
    const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(s.tmap[s.cur]);
    // a programmatic dependent launch: its CTAs may start their source prologue while
    // the previous kernel in the stream finishes (the kernel waits before reading it)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_tiles + A.n_help);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = fused_smem_bytes(g.R);
    cfg.stream = s.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    timing_begin(s);
    cudaError_t e = A.n_help > 0 ? cudaLaunchKernelEx(&cfg, fused2d_kernel<true>, *map, A)
                                 : cudaLaunchKernelEx(&cfg, fused2d_kernel<false>, *map, A);
    timing_end(s);
    s.launches++;
    if (with_cones) s.bin_round++;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

int run_fused_if_supported(Sim &s, int nsteps)
{
    if (s.path == CUE_PATH_PLAIN || s.path == CUE_PATH_PERSIST) return 1;
    if (!fused_supported(s)) {
        if (s.path == CUE_PATH_FUSED) return CUE_ERR_ARG;
        return 1;
    }
    int rc = prepare(s);
    if (rc != CUE_OK) return s.path == CUE_PATH_FUSED ? rc : 1;
    if (nsteps > 0 && s.n_axons > 0 && launch_bin_count(s) != cudaSuccess) return CUE_ERR_CUDA;
    // helpers: sized from the crowding the last run reported (its readback, if landed)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool adapt = s.adapt_helpers && s.n_axons > 0 && s.wl.bin_cap >= s.n_axons &&
                       s.geom.ntx * s.geom.nty <= kHelpMaxTiles &&
                       cudaStreamIsCapturing(s.stream, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone;
    if (adapt && s.help_pending && cudaEventQuery(s.help_ev) == cudaSuccess) {
        // the largest per-launch need of the last run (its last launch's own count too)
        const int need = std::max(s.help_host[0], std::max(s.help_host[1], s.help_host[2]));
        s.help_next = std::min(std::max(need, 0), kMaxHelpers);
        s.help_pending = false;
    }
    const int n_help = adapt ? s.help_next : 0;
    s.help_last = 0;
    while (nsteps > 0) {
        int k = nsteps < s.geom.K ? nsteps : s.geom.K;
        if (launch_fused(s, k, true, n_help) != cudaSuccess) return CUE_ERR_CUDA;
        s.help_last = n_help;
        s.cur ^= 1;
        s.field_step += k;
        s.cone_step += k;
        nsteps -= k;
    }
    if (adapt && !s.help_pending) {     // read this run's last reported need back, without waiting
        if (!s.help_host && cudaHostAlloc(reinterpret_cast<void **>(&s.help_host), 3 * sizeof(int),
                                          cudaHostAllocDefault) != cudaSuccess)
            s.help_host = nullptr;
        if (s.help_host && !s.help_ev && cudaEventCreateWithFlags(&s.help_ev, cudaEventDisableTiming) != cudaSuccess)
            s.help_ev = nullptr;
        if (s.help_host && s.help_ev &&
            cudaMemcpyAsync(s.help_host, s.bin_ctl() + 3, 3 * sizeof(int), cudaMemcpyDeviceToHost, s.stream) ==
                cudaSuccess &&
            cudaEventRecord(s.help_ev, s.stream) == cudaSuccess)
            s.help_pending = true;
    }
    s.fused_used = true;
    return CUE_OK;
}

int field_fused_if_supported(Sim &s, int nsteps)
{
    if (s.path == CUE_PATH_PLAIN || s.path == CUE_PATH_PERSIST) return 1;
    if (!fused_supported(s)) return s.path == CUE_PATH_FUSED ? CUE_ERR_ARG : 1;
    int rc = prepare(s);
    if (rc != CUE_OK) return s.path == CUE_PATH_FUSED ? rc : 1;
    while (nsteps > 0) {
        int k = nsteps < s.geom.K ? nsteps : s.geom.K;
        if (launch_fused(s, k, false) != cudaSuccess) return CUE_ERR_CUDA;
        s.cur ^= 1;
        s.field_step += k;
        nsteps -= k;
    }
    s.fused_used = true;
    return CUE_OK;
}

}  // namespace cue
