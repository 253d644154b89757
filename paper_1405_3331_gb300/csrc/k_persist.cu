// k_persist.cu -- persistent coupled-step engine for 2D grids: one cooperative
// launch runs many steps of one or many simulation instances.
//
// A step of an instance is one phase: its field tiles (C^n -> C^{n+1} with the
// rate map and the point sources) and its cone chunks (cones read C^n) touch
// disjoint outputs, so every block walks one shared work list of (instance,
// item) pairs, then all blocks meet at a grid barrier and the buffers swap.
// The step costs a pass over the list plus one barrier instead of two or three
// kernel launches, which is what a grid that fits in L2 (a few MB) is bound
// by.  The same kernel steps a batch of independent instances of uneven sizes
// and parameters: the per-instance table holds each one's physics, buffers
// and tiling, and the work list holds their items instance by instance.
//
// Arithmetic per node and per cone is the plain path's (node_update2, the map
// as fma(dt, M, C'), sources added after the update; cone_update), so this
// path matches the plain kernels bit for bit for distinct source cells.
//
// Coherence: data written during the launch (field buffers, cone state) is
// read with ld.global.cg (L2), never through the non-coherent read-only path;
// the barrier orders the steps with device-scope fences.  Every wait in the
// barrier is bounded: past the limit the block raises the timeout status and
// sets an abort flag that makes every other block leave at its next barrier.
#include <algorithm>
#include <vector>

#include "cue_barrier.cuh"
#include "cue_internal.h"

namespace cue {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool finite4(const float4 &v)
{
    const float big = 3.402823466e38f;
    return fabsf(v.x) <= big && fabsf(v.y) <= big && fabsf(v.z) <= big && fabsf(v.w) <= big;
}

// ---------------------------------------------------------------- one field tile
// 32 lanes x 4 nodes in x (128 columns), 8 warps x R rows in y: the plain
// float4 field kernel's block, here one work item.  Every load of the strip
// (R + 2 rows, the R rows of the map, the warp-edge columns) is issued before
// the first update, so a tile costs one L2 round trip.  Sources inside the
// tile are added after its update (atomic, so duplicate cells accumulate).
template <int R, bool MAP>
__device__ __forceinline__ void field_tile_r(const PInst &I, const float *Cin, float *Cout, int tile, int src_begin,
                                             int src_n, bool check)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const FieldDesc &f = I.f;
    const int tx = tile % I.ntx, ty = tile / I.ntx;
    const int p4 = I.pitch >> 2;                       // row pitch in float4
    const int nxq = (f.nx + 3) >> 2;                   // float4 groups holding real columns
    const int x4 = tx * 32 + lane;
    const bool xin = x4 < nxq;
    const int y0 = (ty * kPersistWarps + warp) * R;
    const int x = x4 * 4;
    const bool has_l = x > 0, has_r = x + 4 < f.nx;
    const bool ragged = (tx + 1) * 128 > f.nx;          // this tile holds the right wall (tile-uniform)
    const float4 *in4 = reinterpret_cast<const float4 *>(Cin);
    float4 *out4 = reinterpret_cast<float4 *>(Cout);
    const float4 *m4 = reinterpret_cast<const float4 *>(I.map);
    bool bad = false;
    if (y0 < f.ny) {                                   // warp-uniform
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 v[R + 2], m[MAP ? R : 1];
        float el[R], er[R];
        const float4 *col = in4 + x4;
#pragma unroll
        for (int k = 0; k < R + 2; ++k) {              // rows y0 - 1 .. y0 + R (clamped; walls fixed below)
            const int y = min(max(y0 - 1 + k, 0), f.ny - 1);
            v[k] = xin ? __ldcg(col + y * p4) : z4;
        }
        if constexpr (MAP) {
#pragma unroll
            for (int k = 0; k < R; ++k) m[k] = xin ? __ldg(m4 + min(y0 + k, f.ny - 1) * p4 + x4) : z4;
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            el[k] = 0.f;
            er[k] = 0.f;
        }
        if (lane == 0 && xin && has_l) {
#pragma unroll
            for (int k = 0; k < R; ++k) el[k] = __ldcg(Cin + (size_t)min(y0 + k, f.ny - 1) * I.pitch + x - 1);
        }
        if (lane == 31 && xin && has_r) {
#pragma unroll
            for (int k = 0; k < R; ++k) er[k] = __ldcg(Cin + (size_t)min(y0 + k, f.ny - 1) * I.pitch + x + 4);
        }
        // columns x .. x+3: which are real, and which have a real right neighbour
        const bool v1 = !ragged || x + 1 < f.nx, v2 = !ragged || x + 2 < f.nx, v3 = !ragged || x + 3 < f.nx;
        float4 *orow = out4 + x4 + y0 * p4;
        int base = y0 * I.pitch + x;
#pragma unroll
        for (int k = 0; k < R; ++k, orow += p4, base += I.pitch) {
            const int y = y0 + k;
            if (y >= f.ny) break;                      // warp-uniform
            const float4 cur = v[k + 1];
            const float4 up = y > 0 ? v[k] : cur;
            const float4 dn = y + 1 < f.ny ? v[k + 2] : cur;
            float l = __shfl_up_sync(kFull, cur.w, 1);
            float r = __shfl_down_sync(kFull, cur.x, 1);
            if (lane == 0) l = has_l ? el[k] : cur.x;
            if (lane == 31) r = has_r ? er[k] : cur.w;
            if (!has_l) l = cur.x;
            if (!has_r) r = cur.w;
            if (xin) {
                float4 o;
                if (ragged) {
                    // a missing right neighbour (the wall, possibly inside this float4) is the node itself
                    const float rx = v1 ? cur.y : cur.x, ry = v2 ? cur.z : cur.y, rz = v3 ? cur.w : cur.z;
                    o.x = node_update2(cur.x, l, rx, up.x, dn.x, f.alpha, f.beta);
                    o.y = node_update2(cur.y, cur.x, ry, up.y, dn.y, f.alpha, f.beta);
                    o.z = node_update2(cur.z, cur.y, rz, up.z, dn.z, f.alpha, f.beta);
                } else {
                    o.x = node_update2(cur.x, l, cur.y, up.x, dn.x, f.alpha, f.beta);
                    o.y = node_update2(cur.y, cur.x, cur.z, up.y, dn.y, f.alpha, f.beta);
                    o.z = node_update2(cur.z, cur.y, cur.w, up.z, dn.z, f.alpha, f.beta);
                }
                o.w = node_update2(cur.w, cur.z, r, up.w, dn.w, f.alpha, f.beta);
                if constexpr (MAP) {
                    o.x = fmaf(f.dt, m[k].x, o.x);
                    o.y = fmaf(f.dt, m[k].y, o.y);
                    o.z = fmaf(f.dt, m[k].z, o.z);
                    o.w = fmaf(f.dt, m[k].w, o.w);
                }
                // this tile's binned sources at these four nodes, in source order
                for (int e = 0; e < src_n; ++e) {
                    const int2 ent = __ldg(reinterpret_cast<const int2 *>(I.src_ent) + src_begin + e);
                    const int rel = ent.x - base;
                    if (rel >= 0 && rel < 4) {
                        const float em = __ldg(I.src_emit + ent.y);
                        if (rel == 0) o.x += em;
                        else if (rel == 1) o.y += em;
                        else if (rel == 2) o.z += em;
                        else o.w += em;
                    }
                }
                if (ragged) {
                    if (!v1) o.y = cur.y;              // padding columns keep their contents
                    if (!v2) o.z = cur.z;
                    if (!v3) o.w = cur.w;
                }
                if (check) bad |= !finite4(o);
                *orow = o;
            }
        }
    }
    if (check && __any_sync(kFull, bad) && lane == 0) flag_status(I.status, kStatusNonFinite);
    if (src_n < 0) {                                   // sources not binned: scan them, add atomically
        __syncthreads();                               // the tile's stores, visible to the block
        const int bx0 = tx * 128, bx1 = min(bx0 + 128, f.nx);
        const int by0 = ty * kPersistWarps * R, by1 = min(by0 + kPersistWarps * R, f.ny);
        const long long n_cells = (long long)f.nx * f.ny;
        for (int k = threadIdx.x; k < I.n_src; k += blockDim.x) {
            const int c = __ldg(I.src_cell + k);
            if (c < 0 || (long long)c >= n_cells) {
                if (tile == 0) flag_status(I.status, kStatusBounds);
                continue;
            }
            const int cx = c % f.nx, cy = c / f.nx;
            if (cx >= bx0 && cx < bx1 && cy >= by0 && cy < by1)
                atomicAdd(Cout + (size_t)cy * I.pitch + cx, __ldg(I.src_emit + k));
        }
    }
}

// The same tile of I.rows rows per warp (any count), streamed: each warp walks
// its rows down y keeping the rows above, at and below in registers and the
// next row, its edge columns and its map row in flight, so a tile needs few
// registers and many can be resident (the launch-per-step batch mode).  The
// arithmetic, wall handling and source order are field_tile_r's.
template <bool MAP>
__device__ __forceinline__ void field_tile_stream(const PInst &I, const float *Cin, float *Cout, int tile,
                                                  int src_begin, int src_n, bool check)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const FieldDesc &f = I.f;
    const int R = I.rows;
    const int tx = tile % I.ntx, ty = tile / I.ntx;
    const int p4 = I.pitch >> 2;
    const int nxq = (f.nx + 3) >> 2;
    const int x4 = tx * 32 + lane;
    const bool xin = x4 < nxq;
    const int y0 = (ty * kPersistWarps + warp) * R;
    const int x = x4 * 4;
    const bool has_l = x > 0, has_r = x + 4 < f.nx;
    const bool ragged = (tx + 1) * 128 > f.nx;
    const float4 *col = reinterpret_cast<const float4 *>(Cin) + x4;
    float4 *out4 = reinterpret_cast<float4 *>(Cout);
    const float4 *m4 = reinterpret_cast<const float4 *>(I.map);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    bool bad = false;
    if (y0 < f.ny) {                                   // warp-uniform
        const int y1 = min(y0 + R, f.ny);
        auto row = [&](int y) { return xin ? __ldcg(col + (size_t)min(max(y, 0), f.ny - 1) * p4) : z4; };
        const bool need_l = lane == 0 && xin && has_l, need_r = lane == 31 && xin && has_r;
        auto edge_l = [&](int y) { return need_l ? __ldcg(Cin + (size_t)min(y, f.ny - 1) * I.pitch + x - 1) : 0.f; };
        auto edge_r = [&](int y) { return need_r ? __ldcg(Cin + (size_t)min(y, f.ny - 1) * I.pitch + x + 4) : 0.f; };
        auto map_row = [&](int y) {
            return (MAP && xin) ? __ldg(m4 + (size_t)min(y, f.ny - 1) * p4 + x4) : z4;
        };
        float4 vm = row(y0 - 1), vc = row(y0), vp = row(y0 + 1);    // rows y-1, y, y+1 (clamped)
        float el = edge_l(y0), er = edge_r(y0);
        float4 m = map_row(y0);
        const bool v1 = !ragged || x + 1 < f.nx, v2 = !ragged || x + 2 < f.nx, v3 = !ragged || x + 3 < f.nx;
        for (int y = y0; y < y1; ++y) {
            // the next row's inputs go out before this row is computed
            const bool more = y + 1 < y1;
            const float4 vn = more ? row(y + 2) : z4;
            const float eln = more ? edge_l(y + 1) : 0.f, ern = more ? edge_r(y + 1) : 0.f;
            const float4 mn = more ? map_row(y + 1) : z4;
            // rows y - 1 and y + 1 were loaded clamped: at a wall they are row y itself
            const float4 cur = vc, up = vm, dn = vp;
            float l = __shfl_up_sync(kFull, cur.w, 1);
            float r = __shfl_down_sync(kFull, cur.x, 1);
            if (lane == 0) l = has_l ? el : cur.x;     // only lane 0 can lack a left neighbour
            if (lane == 31) r = er;
            if (!has_r) r = cur.w;
            if (xin) {
                float4 o;
                if (ragged) {
                    const float rx = v1 ? cur.y : cur.x, ry = v2 ? cur.z : cur.y, rz = v3 ? cur.w : cur.z;
                    o.x = node_update2(cur.x, l, rx, up.x, dn.x, f.alpha, f.beta);
                    o.y = node_update2(cur.y, cur.x, ry, up.y, dn.y, f.alpha, f.beta);
                    o.z = node_update2(cur.z, cur.y, rz, up.z, dn.z, f.alpha, f.beta);
                } else {
                    o.x = node_update2(cur.x, l, cur.y, up.x, dn.x, f.alpha, f.beta);
                    o.y = node_update2(cur.y, cur.x, cur.z, up.y, dn.y, f.alpha, f.beta);
                    o.z = node_update2(cur.z, cur.y, cur.w, up.z, dn.z, f.alpha, f.beta);
                }
                o.w = node_update2(cur.w, cur.z, r, up.w, dn.w, f.alpha, f.beta);
                if constexpr (MAP) {
                    o.x = fmaf(f.dt, m.x, o.x);
                    o.y = fmaf(f.dt, m.y, o.y);
                    o.z = fmaf(f.dt, m.z, o.z);
                    o.w = fmaf(f.dt, m.w, o.w);
                }
                const int base = y * I.pitch + x;
                for (int e = 0; e < src_n; ++e) {
                    const int2 ent = __ldg(reinterpret_cast<const int2 *>(I.src_ent) + src_begin + e);
                    const int rel = ent.x - base;
                    if (rel >= 0 && rel < 4) {
                        const float em = __ldg(I.src_emit + ent.y);
                        if (rel == 0) o.x += em;
                        else if (rel == 1) o.y += em;
                        else if (rel == 2) o.z += em;
                        else o.w += em;
                    }
                }
                if (ragged) {
                    if (!v1) o.y = cur.y;
                    if (!v2) o.z = cur.z;
                    if (!v3) o.w = cur.w;
                }
                if (check) bad |= !finite4(o);
                out4[(size_t)y * p4 + x4] = o;
            }
            vm = vc;
            vc = vp;
            vp = vn;
            el = eln;
            er = ern;
            m = mn;
        }
    }
    if (check && __any_sync(kFull, bad) && lane == 0) flag_status(I.status, kStatusNonFinite);
    if (src_n < 0) {                                   // sources not binned: scan them, add atomically
        __syncthreads();
        const int bx0 = tx * 128, bx1 = min(bx0 + 128, f.nx);
        const int by0 = ty * kPersistWarps * R, by1 = min(by0 + kPersistWarps * R, f.ny);
        const long long n_cells = (long long)f.nx * f.ny;
        for (int k = threadIdx.x; k < I.n_src; k += blockDim.x) {
            const int c = __ldg(I.src_cell + k);
            if (c < 0 || (long long)c >= n_cells) {
                if (tile == 0) flag_status(I.status, kStatusBounds);
                continue;
            }
            const int cx = c % f.nx, cy = c / f.nx;
            if (cx >= bx0 && cx < bx1 && cy >= by0 && cy < by1)
                atomicAdd(Cout + (size_t)cy * I.pitch + cx, __ldg(I.src_emit + k));
        }
    }
}

// Non-finite values persist once they appear, so the check runs on the last
// step of a launch only (`check`).
__device__ __forceinline__ void field_tile(const PInst &I, const float *Cin, float *Cout, const PItem &w, bool check)
{
    if (I.map) {
        switch (I.rows) {
        case 1: field_tile_r<1, true>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check); break;
        case 2: field_tile_r<2, true>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check); break;
        default: field_tile_r<4, true>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check); break;
        }
    } else {
        switch (I.rows) {
        case 1: field_tile_r<1, false>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check); break;
        case 2: field_tile_r<2, false>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check); break;
        default: field_tile_r<4, false>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check); break;
        }
    }
}

// ---------------------------------------------------------------- one cone chunk
// The cone's state loads are issued together and its noise is drawn while they
// are in flight; the active count goes to a per-thread counter (added to the
// handle's counter once, at the end of the launch).
__device__ __forceinline__ void cone_chunk(const PInst &I, const float *C, int chunk, uint32_t step,
                                           const float *pin, const float *din, float *pout, float *dout,
                                           unsigned &n_live)
{
    const int a = chunk * kPersistConeChunk + threadIdx.x;
    const int n = I.n_axons;
    if (a >= n) return;
    const uint8_t act = __ldcg(I.active + a);
    float p[2], d[2];
    p[0] = __ldcg(pin + a);
    p[1] = __ldcg(pin + n + a);
    d[0] = __ldcg(din + a);
    d[1] = __ldcg(din + n + a);
    float xi[2];
    cone_noise<2>(I.c.key0, I.c.key1, (uint32_t)a, step, xi);
    if (!act) return;
    n_live++;
    const size_t sy = I.pitch;
    auto ld = [&](int i, int j, int) { return __ldcg(C + (size_t)i + sy * j); };
    const bool stop = I.c.stop_r2 >= 0.0f && I.n_src > 0;
    const bool alive = cone_step_rule<2>(I.f, I.c, ld, xi, p, d, I.src_xyz, I.n_src, stop ? I.n_src : 0);
    pout[a] = p[0];
    pout[n + a] = p[1];
    dout[a] = d[0];
    dout[n + a] = d[1];
    if (!alive) I.active[a] = 0;
    const float big = 3.402823466e38f;
    if (!(fabsf(p[0]) <= big && fabsf(p[1]) <= big && fabsf(d[0]) <= big && fabsf(d[1]) <= big))
        flag_status(I.status, kStatusNonFinite);
}

// Add a thread's cone-update count to its instance's counter when the thread
// moves to another instance's cones (and at the end of the launch).
// Called by every thread of the block (block-uniform): one atomic per warp.
__device__ __forceinline__ void flush_live(const PInst *insts, int &live_inst, int next, unsigned &n_live)
{
    if (live_inst == next) return;
    const unsigned tot = __reduce_add_sync(kFull, n_live);
    if (live_inst >= 0 && tot && (threadIdx.x & 31) == 0)
        atomicAdd(insts[live_inst].counter, (unsigned long long)tot);
    n_live = 0;
    live_inst = next;
}

__global__ void __launch_bounds__(kPersistThreads, 3) persist_kernel(const PInst *__restrict__ insts,
                                                                  const PItem *__restrict__ items, int n_items,
                                                                  int nsteps, int cur0, uint32_t step0, PBar *bar,
                                                                  unsigned expected, long long limit,
                                                                  unsigned *status, const PCtrl *ctrl)
{
    if (ctrl) {
        cur0 = ctrl->cur;
        step0 = ctrl->step0;
    }
    unsigned n_live = 0;                               // cone updates by this thread (one instance per item)
    int live_inst = -1;
    for (int s = 0; s < nsteps; ++s) {
        const int cur = (cur0 + s) & 1;
        PItem nxt = (int)blockIdx.x < n_items ? items[blockIdx.x] : PItem{};
        for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
            const PItem w = nxt;
            if (it + (int)gridDim.x < n_items) nxt = items[it + gridDim.x];   // in flight while w runs
            const PInst &I = insts[w.inst];
            const float *Cin;
            float *Cout;
            if (I.traj_field) {                         // trajectory mode: step s reads slot s, writes s + 1
                Cin = I.traj_field + (size_t)s * I.cells;
                Cout = I.traj_field + (size_t)(s + 1) * I.cells;
            } else {
                Cin = cur ? I.field1 : I.field0;
                Cout = cur ? I.field0 : I.field1;
            }
            if (w.idx >= 0) {
                field_tile(I, Cin, Cout, w, s + 1 == nsteps);
            } else if (I.traj_cone) {
                const size_t cn = (size_t)2 * I.n_axons;
                const float *pin = I.traj_cone + (size_t)s * 2 * cn;
                float *pout = I.traj_cone + (size_t)(s + 1) * 2 * cn;
                flush_live(insts, live_inst, w.inst, n_live);
                cone_chunk(I, Cin, ~w.idx, step0 + (uint32_t)s, pin, pin + cn, pout, pout + cn, n_live);
            } else {
                flush_live(insts, live_inst, w.inst, n_live);
                cone_chunk(I, Cin, ~w.idx, step0 + (uint32_t)s, I.pos, I.dir, I.pos, I.dir, n_live);
            }
        }
        if (s + 1 < nsteps && !grid_barrier(bar, expected, limit, status)) break;
    }
    flush_live(insts, live_inst, -1, n_live);
}

// One block per instance: each source's field tile (by the instance's rows),
// then its rank among the (tile, index) keys by counting, which places it in
// the sorted entry list.  Out-of-range cells raise the bounds status and sort
// last with offset -1, never matched.
__global__ void __launch_bounds__(256) bin_sources_kernel(const PInst *__restrict__ insts, unsigned *status)
{
    __shared__ int key[kPersistBinCap];
    const PInst &I = insts[blockIdx.x];
    const int n = I.n_src;
    if (n <= 0 || n > kPersistBinCap || !I.src_ent) return;
    const long long n_cells = (long long)I.f.nx * I.f.ny;
    const int rows_px = kPersistWarps * I.rows;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int c = I.src_cell[k];
        if (c < 0 || (long long)c >= n_cells) {
            key[k] = 0x7fffffff;
            flag_status(I.status, kStatusBounds);
        } else {
            key[k] = (c % I.f.nx) / 128 + I.ntx * ((c / I.f.nx) / rows_px);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int kk = key[k];
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += (key[j] < kk) || (key[j] == kk && j < k);
        const int c = I.src_cell[k];
        PSrc e;
        e.off = kk == 0x7fffffff ? -1 : (c / I.f.nx) * I.pitch + c % I.f.nx;
        e.k = k;
        I.src_ent[rank] = e;
        I.src_key[rank] = kk;
    }
}

// Each field-tile item's range of its instance's binned sources.
__global__ void item_sources_kernel(const PInst *__restrict__ insts, PItem *items, int n_items)
{
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n_items) return;
    PItem w = items[it];
    w.src_begin = 0;
    w.src_n = 0;
    if (w.idx >= 0) {
        const PInst &I = insts[w.inst];
        if (I.n_src > kPersistBinCap || (I.n_src > 0 && !I.src_ent)) {
            w.src_n = -1;
        } else if (I.n_src > 0) {
            int lo = 0, hi = I.n_src;                  // first key >= tile
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (I.src_key[mid] < w.idx) lo = mid + 1;
                else hi = mid;
            }
            int end = lo;
            while (end < I.n_src && I.src_key[end] == w.idx) ++end;
            w.src_begin = lo;
            w.src_n = end - lo;
        }
    }
    items[it] = w;
}

__global__ void persist_advance(PCtrl *ctrl, int nsteps)
{
    ctrl->cur ^= (nsteps & 1);
    ctrl->step0 += (uint32_t)nsteps;
}

// ---------------------------------------------------------------- one step per launch
// The same work items as ordinary launches, for batches: step s of a run is
// one launch over every instance's cone chunks (one chunk per block), then one
// over every instance's field tiles (one tile per block, the tile function and
// binned sources of the persistent kernel).  No grid barrier: the stream orders
// the steps, and the hardware keeps as many small blocks resident as registers
// allow.  Buffers and the Philox step come from the control block plus s, so a
// captured graph replays without new arguments.
// R > 0: field_tile_r<R>; R == 0: the streamed tile of I.rows rows.
template <int R>
__global__ void __launch_bounds__(kPersistThreads, R == 0 ? 6 : 1) step_tiles_kernel(const PInst *__restrict__ insts,
                                                                     const PItem *__restrict__ items, int s,
                                                                     const PCtrl *ctrl, int check)
{
    const PItem w = items[blockIdx.x];
    const PInst &I = insts[w.inst];
    const int cur = (ctrl->cur + s) & 1;
    const float *Cin = cur ? I.field1 : I.field0;
    float *Cout = cur ? I.field0 : I.field1;
    if constexpr (R == 0) {
        if (I.map) field_tile_stream<true>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check != 0);
        else field_tile_stream<false>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check != 0);
    } else {
        if (I.map) field_tile_r<R, true>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check != 0);
        else field_tile_r<R, false>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check != 0);
    }
}

__device__ __forceinline__ void step_chunk(const PInst *insts, const PItem &w, int s, const PCtrl *ctrl)
{
    const PInst &I = insts[w.inst];
    const int cur = (ctrl->cur + s) & 1;
    const float *Cin = cur ? I.field1 : I.field0;
    unsigned n_live = 0;
    cone_chunk(I, Cin, ~w.idx, ctrl->step0 + (uint32_t)s, I.pos, I.dir, I.pos, I.dir, n_live);
    const unsigned tot = __reduce_add_sync(kFull, n_live);
    if (tot && (threadIdx.x & 31) == 0) atomicAdd(I.counter, (unsigned long long)tot);
}

__global__ void __launch_bounds__(kPersistThreads) step_chunks_kernel(const PInst *__restrict__ insts,
                                                                      const PItem *__restrict__ items, int s,
                                                                      const PCtrl *ctrl)
{
    step_chunk(insts, items[blockIdx.x], s, ctrl);
}

// Cone chunks and streamed tiles of one step in one launch, one item per block,
// over the instance-ordered list (each instance's tiles, then its cone chunks):
// blocks start roughly in index order, so an instance's cones gather from rows
// its tiles have just brought into L2.
__global__ void __launch_bounds__(kPersistThreads, 6) step_merged_kernel(const PInst *__restrict__ insts,
                                                                         const PItem *__restrict__ items, int s,
                                                                         const PCtrl *ctrl, int check)
{
    const PItem w = items[blockIdx.x];
    if (w.idx < 0) {
        step_chunk(insts, w, s, ctrl);
        return;
    }
    const PInst &I = insts[w.inst];
    const int cur = (ctrl->cur + s) & 1;
    const float *Cin = cur ? I.field1 : I.field0;
    float *Cout = cur ? I.field0 : I.field1;
    if (I.map) field_tile_stream<true>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check != 0);
    else field_tile_stream<false>(I, Cin, Cout, w.idx, w.src_begin, w.src_n, check != 0);
}

int sm_count_p()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 152;
    }
    return n;
}

}  // namespace

int persist_max_blocks_per_sm()
{
    static int nb = -1;
    if (nb < 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, persist_kernel, kPersistThreads, 0) != cudaSuccess)
            v = 0;
        nb = v;
    }
    return nb;
}

cudaError_t persist_bin_sources(PInst *d_insts, int n_inst, PItem *d_items, int n_items, unsigned *status,
                                cudaStream_t stream)
{
    if (n_inst <= 0 || n_items <= 0) return cudaSuccess;
    bin_sources_kernel<<<n_inst, 256, 0, stream>>>(d_insts, status);
    item_sources_kernel<<<(n_items + 255) / 256, 256, 0, stream>>>(d_insts, d_items, n_items);
    return cudaGetLastError();
}

int persist_tiles(int nx, int ny, int rows)
{
    const int ntx = ((nx + 3) / 4 + 31) / 32;
    const int nty = (ny + kPersistWarps * rows - 1) / (kPersistWarps * rows);
    return ntx * nty;
}

void persist_fill(PInst &I, const FieldDesc &f, int rows, int pitch)
{
    I.rows = rows;
    I.ntx = ((f.nx + 3) / 4 + 31) / 32;
    I.pitch = pitch;
    I.cells = (size_t)pitch * f.ny;
}

// Work list: every instance's cone chunks first (their dependent loads take
// longest), then the field tiles, instances interleaved round-robin so that a
// block's consecutive items come from different instances.
void persist_items(const std::vector<PInst> &insts, std::vector<PItem> &items)
{
    items.clear();
    const int ni = (int)insts.size();
    std::vector<int> ntile(ni), nchunk(ni);
    int maxc = 0, maxt = 0;
    for (int i = 0; i < ni; ++i) {
        const PInst &I = insts[i];
        ntile[i] = persist_tiles(I.f.nx, I.f.ny, I.rows);
        nchunk[i] = (I.n_axons + kPersistConeChunk - 1) / kPersistConeChunk;
        maxc = std::max(maxc, nchunk[i]);
        maxt = std::max(maxt, ntile[i]);
    }
    if (ni > 1) {
        // batches: instance by instance, each instance's cone chunks right after its
        // tiles, so that the cones' field reads and the tiles' shared halo rows find
        // the instance's field still in L2
        for (int i = 0; i < ni; ++i) {
            for (int k = 0; k < ntile[i]; ++k) items.push_back(PItem{i, k, 0, 0});
            for (int k = 0; k < nchunk[i]; ++k) items.push_back(PItem{i, ~k, 0, 0});
        }
        return;
    }
    // one grid: the cone chunks first (their dependent loads overlap the tiles)
    for (int k = 0; k < maxc; ++k)
        for (int i = 0; i < ni; ++i)
            if (k < nchunk[i]) items.push_back(PItem{i, ~k, 0, 0});
    for (int k = 0; k < maxt; ++k)
        for (int i = 0; i < ni; ++i)
            if (k < ntile[i]) items.push_back(PItem{i, k, 0, 0});
}

cudaError_t step_launch(const PInst *d_insts, const PItem *d_chunks, int n_chunks, const PItem *d_tiles,
                        int n_tiles, const PItem *d_mixed, int rows, int nsteps, PCtrl *ctrl, cudaStream_t stream)
{
    for (int s = 0; s < nsteps; ++s) {
        if (rows > 4 && d_mixed && n_chunks + n_tiles > 0) {
            // streamed tiles: every item of the instance-ordered list in one launch
            step_merged_kernel<<<n_chunks + n_tiles, kPersistThreads, 0, stream>>>(d_insts, d_mixed, s, ctrl,
                                                                                   s + 1 == nsteps);
            continue;
        }
        if (n_chunks > 0) step_chunks_kernel<<<n_chunks, kPersistThreads, 0, stream>>>(d_insts, d_chunks, s, ctrl);
        if (n_tiles > 0) {
            const int check = s + 1 == nsteps;
            if (rows == 1) step_tiles_kernel<1><<<n_tiles, kPersistThreads, 0, stream>>>(d_insts, d_tiles, s, ctrl, check);
            else if (rows == 2)
                step_tiles_kernel<2><<<n_tiles, kPersistThreads, 0, stream>>>(d_insts, d_tiles, s, ctrl, check);
            else if (rows == 4)
                step_tiles_kernel<4><<<n_tiles, kPersistThreads, 0, stream>>>(d_insts, d_tiles, s, ctrl, check);
            else step_tiles_kernel<0><<<n_tiles, kPersistThreads, 0, stream>>>(d_insts, d_tiles, s, ctrl, check);
        }
    }
    persist_advance<<<1, 1, 0, stream>>>(ctrl, nsteps);
    return cudaGetLastError();
}

cudaError_t persist_launch(const PInst *d_insts, const PItem *d_items, int n_items, int nsteps, int cur0,
                           uint32_t step0, PBar *d_bar, int blocks_per_sm, int phantom, long long limit,
                           unsigned *status, cudaStream_t stream, int *grid_out, PCtrl *ctrl)
{
    const int maxb = persist_max_blocks_per_sm();
    if (maxb <= 0) return cudaErrorInvalidConfiguration;
    int bpsm = blocks_per_sm > 0 ? std::min(blocks_per_sm, maxb) : std::min(2, maxb);
    int grid = std::min(n_items, bpsm * sm_count_p());
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = grid;
    cudaError_t e = cudaMemsetAsync(d_bar, 0, sizeof(PBar), stream);
    if (e != cudaSuccess) return e;
    const unsigned expected = (unsigned)grid + (unsigned)(phantom > 0 ? phantom : 0);
    const long long lim = limit > 0 ? limit : kPersistSpinLimit;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kPersistThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;     // all blocks co-resident: the barrier cannot starve
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, persist_kernel, d_insts, d_items, n_items, nsteps, cur0, step0, d_bar, expected,
                           lim, status, static_cast<const PCtrl *>(ctrl));
    if (e != cudaSuccess || !ctrl) return e;
    persist_advance<<<1, 1, 0, stream>>>(ctrl, nsteps);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- single simulation
bool persist_supported(const Sim &s)
{
    return s.fd.dim == 2 && s.vec4 && persist_max_blocks_per_sm() > 0;
}

static int pick_rows(const Sim &s)
{
    if (s.persist_rows > 0) return std::min(s.persist_rows, 4);
    // the longest strips that still give every SM a tile
    const int target = sm_count_p();
    int rows = 4;
    while (rows > 1 && persist_tiles(s.fd.nx, s.fd.ny, rows) < target) rows /= 2;
    return rows;
}

static PInst sim_instance(const Sim &s, int rows)
{
    PInst I{};
    I.f = s.fd;
    I.c = s.cd;
    I.field0 = s.field[0];
    I.field1 = s.field[1];
    I.map = s.src_map;
    I.src_cell = s.src_cell;
    I.src_emit = s.src_emit;
    I.src_xyz = s.src_xyz();
    I.n_src = s.n_src;
    I.pos = s.pos;
    I.dir = s.dir;
    I.active = s.active;
    I.n_axons = s.n_axons;
    I.status = s.status();
    I.counter = s.cone_counter();
    I.src_ent = s.n_src > 0 ? s.persist_src_ent() : nullptr;
    I.src_key = s.n_src > 0 ? s.persist_src_key() : nullptr;
    persist_fill(I, s.fd, rows, s.fd.nx);
    return I;
}

// Upload the instance record and the work list into the workspace (once per
// configuration; the trajectory variant is built per call).
static int persist_prepare(Sim &s, const PInst &I, int slot)
{
    std::vector<PInst> v{I};
    std::vector<PItem> items;
    persist_items(v, items);
    if ((size_t)items.size() > s.wl.persist_items_cap) return CUE_ERR_WORKSPACE;
    PInst *d_inst = s.persist_inst() + slot;
    if (cudaMemcpyAsync(d_inst, &v[0], sizeof(PInst), cudaMemcpyHostToDevice, s.stream) != cudaSuccess ||
        cudaMemcpyAsync(s.persist_items(), items.data(), sizeof(PItem) * items.size(), cudaMemcpyHostToDevice,
                        s.stream) != cudaSuccess ||
        persist_bin_sources(d_inst, 1, s.persist_items(), (int)items.size(), s.status(), s.stream) != cudaSuccess)
        return CUE_ERR_CUDA;
    s.persist_n_items = (int)items.size();
    return CUE_OK;
}

int run_persist_if_supported(Sim &s, int nsteps)
{
    if (s.path != CUE_PATH_AUTO && s.path != CUE_PATH_PERSIST) return 1;
    if (!persist_supported(s)) return s.path == CUE_PATH_PERSIST ? CUE_ERR_ARG : 1;
    if (nsteps <= 0) return CUE_OK;
    if (s.cd.stop_r2 >= 0.0f && s.n_src > 0 && !s.src_xyz_ready) {
        if (launch_src_xyz(s) != cudaSuccess) return CUE_ERR_CUDA;
        s.src_xyz_ready = true;
    }
    const int rows = pick_rows(s);
    if (!s.persist_ready || s.persist_rows_used != rows) {
        int rc = persist_prepare(s, sim_instance(s, rows), 0);
        if (rc != CUE_OK) return rc;
        s.persist_ready = true;
        s.persist_rows_used = rows;
    }
    for (int done = 0; done < nsteps;) {                // launches of at most kPersistMaxSteps steps
        const int k = std::min(nsteps - done, kPersistMaxSteps);
        timing_begin(s);
        cudaError_t e = persist_launch(s.persist_inst(), s.persist_items(), s.persist_n_items, k, s.cur,
                                       (uint32_t)s.cone_step, s.persist_bar(), s.persist_bpsm, s.persist_phantom,
                                       s.persist_limit, s.status(), s.stream, &s.persist_grid);
        timing_end(s);
        s.launches++;
        if (e != cudaSuccess) return CUE_ERR_CUDA;
        s.cur ^= (k & 1);
        s.field_step += k;
        s.cone_step += k;
        done += k;
    }
    s.persist_used = true;
    return CUE_OK;
}

// nsteps coupled steps from (C, p, d) at traj slot 0, storing every step's
// field and cone state in the trajectory buffers (the adjoint's recompute).
int run_persist_trajectory(Sim &s, float *traj_field, float *traj_cone, uint32_t step0, int nsteps)
{
    if (!persist_supported(s)) return 1;
    const int rows = pick_rows(s);
    PInst I = sim_instance(s, rows);
    I.traj_field = traj_field;
    I.traj_cone = traj_cone;
    int rc = persist_prepare(s, I, 1);
    if (rc != CUE_OK) return rc;
    s.persist_ready = false;                            // the work list was overwritten
    cudaError_t e = persist_launch(s.persist_inst() + 1, s.persist_items(), s.persist_n_items, nsteps, 0, step0,
                                   s.persist_bar(), s.persist_bpsm, 0, s.persist_limit, s.status(), s.stream,
                                   nullptr);
    s.launches++;
    return e == cudaSuccess ? CUE_OK : CUE_ERR_CUDA;
}

}  // namespace cue
