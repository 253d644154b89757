// k_blocked.cu -- the temporally blocked batch mode: one launch advances every
// instance of a batch K steps (field and cones, rows a1-a6 of each), one
// HBM round trip of each instance's field per launch.
//
// The work list holds one item per (instance, field tile).  Tiles are aligned
// to the instance's walls (AxisTiles): a tile that holds a wall carries no halo
// beyond it, so an instance up to 256 columns wide is one tile column and one
// up to 94 rows high one tile row.  A CTA loads its
// tile plus a halo from the instance's current buffer with one TMA tensor copy
// (the instance's tensor maps live in the instance table in global memory;
// rows are the instance's pitch apart, columns past nx read as zeros), runs K
// sub-steps in shared memory -- the tile's cones on C^{n+j}, then the in-place
// sweep of the field to C^{n+j+1} (cue_tile.cuh) with the rate map and the
// point sources -- and stores the interior into the other buffer.  This is
// the single-field fused kernel (k_fused.cu) generalised to a table of
// instances of uneven sizes: right x walls may fall inside a float4 group
// (nx % 4 != 0), and a dense rate map is read from global memory per row.
//
// Cones: every tile has a bin that can hold all of its instance's cones, so
// none ever spills, however the cones cluster; the first 512 ids of a bin ride
// in registers for the launch, the rest are stepped from global memory.  Each
// launch re-bins its cones into the other round of bins as they finish; each
// tile clears its own count once read.
//
// Step control: the buffer parity, the Philox step and the bin round are read
// from the batch's control block at the start of the launch, and the last CTA
// to finish advances them, so a captured graph replays without new arguments.
// A launch writes its K steps' result into the other buffer, so the current
// buffer flips once per launch (not once per step as in the other modes).
//
// Arithmetic per node and per cone is the plain path's (node_update2, the map
// as fma(dt, M, C') after the stencil, sources after that; the cone step of
// cue_device.cuh), so every instance matches the plain kernels bit for bit for
// distinct source cells.  Model: cue field on an Eulerian grid (Sec. 5.2) with
// sources of their own rates (Sec. 4.3); cone steering by vector addition
// (Sec. 3.5, Eq. 6-7) with stateless counter-based noise (Sec. 5.1) and
// Box-Muller (Sec. 3.2); stop tests on the bounds (Sec. 3.4) and squared
// source distance (Sec. 3.3).
#include <cuda.h>

#include <algorithm>
#include <cmath>

#include "cue_internal.h"
#include "cue_tile.cuh"

namespace cue {
static_assert(kBlockedTileW == tile::kW && kBlockedTileRows == tile::kRows && kBlockedThreads == tile::kThreads,
              "blocked tile shape");

namespace {

using namespace tile;

constexpr int kConeSlots = 2;          // cones held in registers per thread (kFusedBinCap ids)

struct BlockedArgs {
    const BInst *insts;
    const int2 *items;                 // (instance, tile of the instance)
    PCtrl *ctrl;                       // cur, step0, bin round (pad[0]); advanced by the last CTA
    int K;                             // sub-steps of this launch
    int *counts;                       // [2][total_tiles]
    int *ids;                          // [2][bin_total]
    size_t bin_total;
    int total_tiles;
    int *done;                         // CTAs finished (the last resets it and advances ctrl)
    unsigned *status;
};

__device__ __forceinline__ int tile_of_b(const BInst &I, float px, float py)
{
    const FieldDesc &f = I.f;
    int ix = clampi((int)floorf(px * f.inv_h), 0, f.nx - 1);
    int iy = clampi((int)floorf(py * f.inv_h), 0, f.ny - 1);
    return blocked_y(I.g, f.ny).index(iy) * I.g.ntx + blocked_x(I.g, f.nx).index(ix);
}

// The first `real` (>= 1) components of a group are finite (the rest is row padding).
__device__ __forceinline__ bool finite_upto(const float4 &v, int real)
{
    const float big = 3.4e38f;
    return fabsf(v.x) <= big && (real < 2 || fabsf(v.y) <= big) && (real < 3 || fabsf(v.z) <= big) &&
           (real < 4 || fabsf(v.w) <= big);
}

__global__ void __launch_bounds__(kThreads, 2) blocked_kernel(const BlockedArgs A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // layout: mbarrier at 0; the TMA tile at 128 (128-byte aligned); then the lists
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    float *S = reinterpret_cast<float *>(smem_raw + 128);
    float4 *S4 = reinterpret_cast<float4 *>(smem_raw + 128);
    int *row_start = reinterpret_cast<int *>(S + kRows * kW);    // R + 1
    int *row_fill = row_start + (kRows + 1);                      // R
    int *t_col = row_fill + kRows;                                // kBlockedMaxSrc each:
    int *t_row = t_col + kBlockedMaxSrc;
    float *t_e = reinterpret_cast<float *>(t_row + kBlockedMaxSrc);
    float *t_xy = t_e + kBlockedMaxSrc;                          // [2][kBlockedMaxSrc] tile sources
    int *cid = reinterpret_cast<int *>(t_xy + 2 * kBlockedMaxSrc);   // [kThreads] slot-0 cone ids
    float *nzb = reinterpret_cast<float *>(cid + kThreads);       // [2 parity][2][kThreads] noise

    const int2 item = A.items[blockIdx.x];
    const BInst &I = A.insts[item.x];
    const FieldDesc &f = I.f;
    const ConeDesc &c = I.c;
    const FusedGeom &g = I.g;
    const int t = item.y;
    const int gt = I.tile_base + t;
    const int tx = t % g.ntx, ty = t / g.ntx;
    const AxisTiles ax = blocked_x(g, f.nx), ay = blocked_y(g, f.ny);
    const int ox = ax.origin(tx), oy = ay.origin(ty);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = I.n_axons;

    // a programmatic dependent launch: the next launch's CTAs may be scheduled as this
    // launch's CTAs finish.  Up to griddepcontrol.wait a CTA reads only what no kernel
    // writes (the instance table, the point sources), so that part of its prologue
    // overlaps the previous launch's last tiles; the wait (a no-op without the launch
    // attribute) returns once the previous launch has completed and its writes (step
    // control, fields, cone bins and state) are visible.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) mbar_init(bar, 1);
    for (int r = tid; r < kRows; r += kThreads) row_fill[r] = 0;
    __syncthreads();
    // point sources inside the loaded region, grouped by tile row
    const bool stop_on = c.stop_r2 >= 0.0f && I.n_src > 0;
    for (int s = tid; s < I.n_src; s += kThreads) {
        int cell = I.src_cell[s];
        if (cell >= 0 && cell < f.nx * f.ny) {
            int gx = cell % f.nx, gy = cell / f.nx;
            if (gx >= ox && gx < ox + kW && gy >= oy && gy < oy + kRows) atomicAdd(&row_fill[gy - oy], 1);
        } else if (t == 0) {
            flag_status(A.status, kStatusBounds);      // skipped, reported by the instance's first tile
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
    for (int r = tid; r < kRows; r += kThreads) row_fill[r] = 0;
    __syncthreads();
    for (int s = tid; s < I.n_src; s += kThreads) {
        int cell = I.src_cell[s];
        if (cell >= 0 && cell < f.nx * f.ny) {
            int gx = cell % f.nx, gy = cell / f.nx;
            if (gx >= ox && gx < ox + kW && gy >= oy && gy < oy + kRows) {
                int r = gy - oy;
                int slot = row_start[r] + atomicAdd(&row_fill[r], 1);
                t_col[slot] = gx - ox;
                t_row[slot] = r;
                t_e[slot] = I.src_emit[s];
                t_xy[slot] = (float)gx * f.h;
                t_xy[kBlockedMaxSrc + slot] = (float)gy * f.h;
            }
        }
    }

    // from here on: what earlier launches wrote
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int cur = A.ctrl->cur;
    const uint32_t step0 = A.ctrl->step0;
    const int round = (int)A.ctrl->pad[0] & 1;
    if (tid == 0) {
        // the tensor map lives in global memory (written before the launch): make it
        // visible to the tensor-map proxy before the copy uses it
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&I.map[cur]) : "memory");
        mbar_expect_tx(bar, (unsigned)(kRows * kW * sizeof(float)));
        tma_load_2d(S, &I.map[cur], bar, ox, oy);
    }

    // this tile's cones into registers (overlaps the TMA load)
    int *cnt_cur = A.counts + (size_t)round * A.total_tiles;
    int *cnt_next = A.counts + (size_t)(round ^ 1) * A.total_tiles;
    const int *bin = A.ids + (size_t)round * A.bin_total + I.bin_base + (size_t)t * n;
    int *ids_next = A.ids + (size_t)(round ^ 1) * A.bin_total + I.bin_base;
    const int n_bin = n > 0 ? min(cnt_cur[gt], n) : 0;
    int ca[kConeSlots];
    bool cl[kConeSlots];
    float cp[kConeSlots][2], cdir[kConeSlots][2];
#pragma unroll
    for (int q = 0; q < kConeSlots; ++q) {
        int i = tid + q * kThreads;
        ca[q] = i < n_bin ? bin[i] : -1;
        cl[q] = ca[q] >= 0;
        if (cl[q]) {
            cl[q] = I.active[ca[q]] != 0;
            cp[q][0] = I.pos[ca[q]];
            cp[q][1] = I.pos[n + ca[q]];
            cdir[q][0] = I.dir[ca[q]];
            cdir[q][1] = I.dir[n + ca[q]];
        }
    }
    // noise of the slot-0 cones drawn one sub-step ahead by the threads that hold
    // no cone; the first sub-step's here, while the tile copy is in flight
    const int cnt0 = min(n_bin, kThreads);
    const bool pre_noise = cnt0 > 0 && cnt0 <= kThreads - 64;
    cid[tid] = ca[0];
    if (pre_noise && ca[0] >= 0) {
        float xi[2];
        cone_noise<2>(c.key0, c.key1, (uint32_t)ca[0], step0, xi);
        nzb[tid] = xi[0];
        nzb[kThreads + tid] = xi[1];
    }

    __syncthreads();
    if (tid == 0 && n > 0) cnt_cur[gt] = 0;           // read by every thread: cleared for the launch after next
    // the last CTA to finish advances the step control (every CTA read it at its start)
    auto finish = [&]() {
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            if (atomicAdd(A.done, 1) == (int)gridDim.x - 1) {
                __threadfence();
                PCtrl *ctl = A.ctrl;
                ctl->cur = cur ^ 1;             // K steps in shared memory, one buffer flip
                ctl->step0 = step0 + (uint32_t)A.K;
                ctl->pad[0] = (uint32_t)(round ^ 1);
                *A.done = 0;
            }
        }
    };

    // wait for the tile: one thread polls (bounded), the rest wait at the barrier
    bool ok = true;
    if (tid == 0) ok = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            flag_status(A.status, kStatusTimeout);
            mbar_wait_bounded(bar, 0);      // let an in-flight copy land before the CTA exits
        }
        finish();
        return;
    }
    mbar_wait_bounded(bar, 0);              // completed phase: returns at once, acquires the tile

    const int r0 = warp * kBand;
    const int colA = 4 * lane, colB = 128 + 4 * lane;
    const int gxA = ox + colA, gxB = ox + colB;
    const float2 alpha2 = make_float2(f.alpha, f.alpha), beta2 = make_float2(f.beta, f.beta);
    const BandSources bsrc{t_col, t_row, t_e, row_start[r0], row_start[r0 + kBand]};
    const float *stop_xy = g.local_stop ? t_xy : I.src_xyz;
    const int stop_stride = g.local_stop ? kBlockedMaxSrc : I.n_src;
    const int n_stop = stop_on ? (g.local_stop ? row_start[kRows] : I.n_src) : 0;
    const LaneWalls lw = lane_walls(gxA, gxB, f.nx);
    // the right wall inside a group on this tile (nx % 4 != 0): the ragged sweep
    const bool ragged = (f.nx & 3) != 0 && ox + kW > f.nx - 1;
    const BandMap bmap{I.rate_map, I.pitch, oy, f.ny, gxA, gxB, f.dt};
    const bool has_map = I.rate_map != nullptr;
    const int gtop = (oy <= -1) ? -oy - 1 : -1;                     // tile row of global y = -1
    const int gbot = (oy + kRows - 1 >= f.ny) ? f.ny - oy : -1;     // tile row of global y = ny
    const bool wall = gtop >= 0 || gbot >= 0;
    if (wall) {       // ghost rows take the edge rows before the first sub-step
        if (gtop >= 0)
            for (int cc = tid; cc < kW; cc += kThreads) S[gtop * kW + cc] = S[(gtop + 1) * kW + cc];
        if (gbot >= 0 && gbot < kRows)
            for (int cc = tid; cc < kW; cc += kThreads) S[gbot * kW + cc] = S[(gbot - 1) * kW + cc];
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
    // one cone step on the shared-memory field (the plain kernel's arithmetic)
    auto step_cone = [&](uint32_t a, uint32_t stp, float *p, float *d, const float *xi_in) {
        int lo[2];
        float fr[2], v[kPatch2], gr[2], xi[2];
        cell_of<2>(f, p, lo, fr);
        const bool inside = max(lo[0] - 1, 0) - ox >= 0 && min(lo[0] + 2, f.nx - 1) - ox < kW &&
                            max(lo[1] - 1, 0) - oy >= 0 && min(lo[1] + 2, f.ny - 1) - oy < kRows;
        if (inside) gather2(f, lo, ld_fast, v);
        else gather2(f, lo, ld, v);
        grad2(c, v, fr, gr);
        if (xi_in) {
            xi[0] = xi_in[0];
            xi[1] = xi_in[1];
        } else {
            cone_noise<2>(c.key0, c.key1, a, stp, xi);
        }
        return cone_finish_xi<2>(c, gr, xi, p, d, stop_xy, stop_stride, n_stop);
    };

    bool stopped[kConeSlots];
#pragma unroll
    for (int q = 0; q < kConeSlots; ++q) stopped[q] = false;

    for (int j = 0; j < A.K; ++j) {
        const uint32_t step = step0 + j;
        // ---- phase A: cones of this tile read C^{n+j}
        if (pre_noise && tid >= cnt0 && j + 1 < A.K) {     // free threads: next sub-step's noise
            float *nz_next = nzb + ((j + 1) & 1) * 2 * kThreads;
            for (int i = tid - cnt0; i < cnt0; i += kThreads - cnt0) {
                float xi[2];
                cone_noise<2>(c.key0, c.key1, (uint32_t)cid[i], step + 1, xi);
                nz_next[i] = xi[0];
                nz_next[kThreads + i] = xi[1];
            }
        }
#pragma unroll
        for (int q = 0; q < kConeSlots; ++q) {
            count_active(I.counter, cl[q]);
            if (cl[q]) {
                float xi_pre[2];
                const float *xi_in = nullptr;
                if (q == 0 && pre_noise) {
                    const float *nz = nzb + (j & 1) * 2 * kThreads;
                    xi_pre[0] = nz[tid];
                    xi_pre[1] = nz[kThreads + tid];
                    xi_in = xi_pre;
                }
                bool alive = step_cone((uint32_t)ca[q], step, cp[q], cdir[q], xi_in);
                if (!alive) {
                    cl[q] = false;
                    stopped[q] = true;
                }
            }
        }
        // cones of the bin beyond the register slots: state through global memory
        // software-pipelined: the next round's cone state (and the ids two rounds ahead)
        // are loaded while this round's cone steps, so a crowded tile is bound by its
        // arithmetic rather than by chains of dependent loads
        if (n_bin > kFusedBinCap) {
            auto id_at = [&](int i) { return i < n_bin ? bin[i] : -1; };
            int a_nn = id_at(kFusedBinCap + kThreads + tid);
            int a_n = id_at(kFusedBinCap + tid);
            bool live_n = a_n >= 0 && I.active[a_n] != 0;
            float p_n[2] = {0.f, 0.f}, d_n[2] = {0.f, 0.f};
            if (live_n) {
                p_n[0] = I.pos[a_n];
                p_n[1] = I.pos[n + a_n];
                d_n[0] = I.dir[a_n];
                d_n[1] = I.dir[n + a_n];
            }
            for (int base = kFusedBinCap; base < n_bin; base += kThreads) {
                const int a = a_n;
                const bool live = live_n;
                float p[2] = {p_n[0], p_n[1]}, d[2] = {d_n[0], d_n[1]};
                a_n = a_nn;                                   // next round: state in flight now
                a_nn = id_at(base + 2 * kThreads + tid);        // the round after next
                live_n = a_n >= 0 && I.active[a_n] != 0;
                if (live_n) {
                    p_n[0] = I.pos[a_n];
                    p_n[1] = I.pos[n + a_n];
                    d_n[0] = I.dir[a_n];
                    d_n[1] = I.dir[n + a_n];
                }
                count_active(I.counter, live);             // warp-uniform trip count
                if (live) {
                    bool alive = step_cone((uint32_t)a, step, p, d, nullptr);
                    I.pos[a] = p[0];
                    I.pos[n + a] = p[1];
                    I.dir[a] = d[0];
                    I.dir[n + a] = d[1];
                    if (!alive) I.active[a] = 0;
                }
            }
        }
        // rows just outside this warp's band, read before anyone overwrites them
        const Row above = ld_row(S4, r0 > 0 ? r0 - 1 : r0, lane);
        const Row below = ld_row(S4, r0 + kBand < kRows ? r0 + kBand : r0 + kBand - 1, lane);
        __syncthreads();
        // ---- phase B: in-place sweep of the band to C^{n+j+1}
        if (has_map) {
            if (wall) {
                if (ragged) sweep_band<true, true, true>(S4, lane, r0, above, below, lw, alpha2, beta2, bsrc, oy, f.ny, bmap);
                else sweep_band<true, false, true>(S4, lane, r0, above, below, lw, alpha2, beta2, bsrc, oy, f.ny, bmap);
            } else {
                if (ragged) sweep_band<false, true, true>(S4, lane, r0, above, below, lw, alpha2, beta2, bsrc, oy, f.ny, bmap);
                else sweep_band<false, false, true>(S4, lane, r0, above, below, lw, alpha2, beta2, bsrc, oy, f.ny, bmap);
            }
        } else {
            if (wall) {
                if (ragged) sweep_band<true, true, false>(S4, lane, r0, above, below, lw, alpha2, beta2, bsrc, oy, f.ny, bmap);
                else sweep_band<true, false, false>(S4, lane, r0, above, below, lw, alpha2, beta2, bsrc, oy, f.ny, bmap);
            } else {
                if (ragged) sweep_band<false, true, false>(S4, lane, r0, above, below, lw, alpha2, beta2, bsrc, oy, f.ny, bmap);
                else sweep_band<false, false, false>(S4, lane, r0, above, below, lw, alpha2, beta2, bsrc, oy, f.ny, bmap);
            }
        }
        __syncthreads();
    }

    // ---- cones back to global memory, binned for the next launch
    auto rebin = [&](int a, float px, float py) {
        const int tl = tile_of_b(I, px, py);
        const int slot = atomicAdd(&cnt_next[I.tile_base + tl], 1);
        if (slot < n) ids_next[(size_t)tl * n + slot] = a;     // a bin holds every cone of its instance
    };
#pragma unroll
    for (int q = 0; q < kConeSlots; ++q) {
        const int a = ca[q];
        if (a < 0) continue;
        I.pos[a] = cp[q][0];
        I.pos[n + a] = cp[q][1];
        I.dir[a] = cdir[q][0];
        I.dir[n + a] = cdir[q][1];
        if (stopped[q]) I.active[a] = 0;
        if (cl[q]) rebin(a, cp[q][0], cp[q][1]);
    }
    for (int i = kFusedBinCap + tid; i < n_bin; i += kThreads) {
        const int a = bin[i];
        if (I.active[a]) rebin(a, I.pos[a], I.pos[n + a]);
    }

    // ---- store the interior: columns below nx (the row padding past the right
    // wall keeps its contents, as on the other paths)
    float *Cout = I.field[cur ^ 1];
    bool bad = false;
    auto put = [&](float *row, int gx, const float4 &v) {
        const int real = f.nx - gx;
        bad |= !finite_upto(v, real);
        if (real >= 4) {
            reinterpret_cast<float4 *>(row)[gx >> 2] = v;
        } else {
            row[gx] = v.x;
            if (real > 1) row[gx + 1] = v.y;
            if (real > 2) row[gx + 2] = v.z;
        }
    };
    // (the interior [ax.start, ax.end) x [ay.start, ay.end) of this tile, inside the grid)
    const int cx0 = ax.start(tx) - ox, cx1 = ax.end(tx) - ox;
    for (int r = ay.start(ty) - oy + warp; r < ay.end(ty) - oy; r += kWarps) {
        float *row = Cout + (size_t)(oy + r) * I.pitch;
        if (colA >= cx0 && colA < cx1) put(row, gxA, S4[r * (kW / 4) + lane]);
        if (colB >= cx0 && colB < cx1) put(row, gxB, S4[r * (kW / 4) + 32 + lane]);
    }
    if (__any_sync(kFull, bad) && lane == 0) flag_status(A.status, kStatusNonFinite);
    finish();
}

// Start of a run: every active cone of every instance into its tile's bin of
// the current round (the counts of both rounds are zero).
__global__ void __launch_bounds__(256) blocked_bin_kernel(const BInst *__restrict__ insts, const int2 *chunks,
                                                          int *counts, int *ids, size_t bin_total, int total_tiles,
                                                          const PCtrl *ctrl)
{
    const int2 ch = chunks[blockIdx.x];            // (instance, first cone)
    const BInst &I = insts[ch.x];
    const int a = ch.y + threadIdx.x;
    const int n = I.n_axons;
    if (a >= n || !I.active[a]) return;
    const int round = (int)ctrl->pad[0] & 1;
    const int tl = tile_of_b(I, I.pos[a], I.pos[n + a]);
    const int slot = atomicAdd(&counts[(size_t)round * total_tiles + I.tile_base + tl], 1);
    if (slot < n) ids[(size_t)round * bin_total + I.bin_base + (size_t)tl * n + slot] = a;
}

}  // namespace

bool blocked_geometry(const FieldDesc &f, float step_len, float stop_r2, bool cones, int K, FusedGeom &g)
{
    if (!fused_geometry(f, step_len, stop_r2, cones, K, g)) return false;
    g.ntx = blocked_x(g, f.nx).count();
    g.nty = blocked_y(g, f.ny).count();
    return true;
}

size_t blocked_smem_bytes()
{
    return 128 + (size_t)kRows * kW * sizeof(float) + sizeof(int) * (2 * kRows + 1) + sizeof(int) * 2 * kBlockedMaxSrc +
           sizeof(float) * 3 * kBlockedMaxSrc + sizeof(int) * kThreads + sizeof(float) * 4 * kThreads;
}

cudaError_t blocked_prepare()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(blocked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)blocked_smem_bytes());
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t blocked_bin(const BInst *d_insts, const int2 *d_chunks, int n_chunks, int *counts, int *ids,
                        size_t bin_total, int total_tiles, const PCtrl *ctrl, cudaStream_t stream)
{
    if (n_chunks <= 0) return cudaSuccess;
    blocked_bin_kernel<<<n_chunks, 256, 0, stream>>>(d_insts, d_chunks, counts, ids, bin_total, total_tiles, ctrl);
    return cudaGetLastError();
}

cudaError_t blocked_launch(const BInst *d_insts, const int2 *d_items, int n_items, int K, PCtrl *ctrl, int *counts,
                           int *ids, size_t bin_total, int total_tiles, int *done, unsigned *status,
                           cudaStream_t stream)
{
    if (n_items <= 0) return cudaSuccess;
    cudaError_t e = blocked_prepare();
    if (e != cudaSuccess) return e;
    BlockedArgs A;
    A.insts = d_insts;
    A.items = d_items;
    A.ctrl = ctrl;
    A.K = K;
    A.counts = counts;
    A.ids = ids;
    A.bin_total = bin_total;
    A.total_tiles = total_tiles;
    A.done = done;
    A.status = status;
    // a programmatic dependent launch (see the kernel's prologue); inside a stream
    // capture it becomes a programmatic edge of the graph
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_items);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = blocked_smem_bytes();
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, blocked_kernel, A);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace cue
