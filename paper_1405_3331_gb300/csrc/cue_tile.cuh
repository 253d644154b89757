// cue_tile.cuh -- the shared-memory tile machinery of the temporally blocked
// 2D kernels (the single-field fused kernel, k_fused.cu, and the batched
// blocked kernel, k_blocked.cu): mbarrier / TMA helpers, and the in-place
// sweep of a warp's band of rows that advances a tile of the field one step.
//
// A tile is kW = 256 loaded columns x kRows = 96 loaded rows of FP32 in shared
// memory, row-major.  Each of the 8 warps owns a band of kBand = 12 rows; a
// lane holds columns 4*lane .. +3 (group a) and 128 + 4*lane .. +3 (group b) of
// a row, x neighbours come by warp shuffle.  The update is the plain kernels'
// node update (node_update2: fma(alpha, (x- + x+) + (y- + y+), beta C)) with a
// missing neighbour at a wall replaced by the node itself, so every path rounds
// identically.  Model: the cue field on the Eulerian grid of Sec. 5.2.
#pragma once

#include <cuda.h>

#include "cue_device.cuh"

namespace cue {
namespace tile {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kW = 256;               // loaded columns per tile: a warp spans a row, 2 float4 per lane
constexpr int kThreads = 256;         // 8 warps
constexpr int kWarps = kThreads / 32;
constexpr long long kWaitLimit = 1LL << 22;
constexpr int kBand = 12;             // rows swept by each warp per sub-step
constexpr int kRows = kWarps * kBand; // loaded rows per tile (96)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after kWaitLimit polls instead of hanging the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase)
{
    for (long long i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// One 2D tensor tile into shared memory.  `map` may live in kernel parameters
// or in global memory (written before the launch); x must be a multiple of 4
// floats (16 bytes), negative or out-of-range coordinates read zeros.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

struct Row {
    float4 a, b;   // columns 4*lane .. +3 and 128 + 4*lane .. +3 of the tile
};

__device__ __forceinline__ Row ld_row(const float4 *S4, int r, int lane)
{
    return Row{S4[r * (kW / 4) + lane], S4[r * (kW / 4) + 32 + lane]};
}

__device__ __forceinline__ void st_row(float4 *S4, int r, int lane, const Row &v)
{
    S4[r * (kW / 4) + lane] = v.a;
    S4[r * (kW / 4) + 32 + lane] = v.b;
}

// New values of a 4-node group from its old values and neighbours, with the
// arithmetic of node_update2: horizontal pairs summed as scalars, the rest two
// nodes at a time with the packed FP32x2 instructions (each lane of a pair
// rounds exactly like the scalar form).  rw (RAGGED only): index 0..2 of the
// node inside the group that lies on the right x wall (its right neighbour is
// itself; a wall on index 3 comes in through R); the nodes past it are padding.
template <bool RAGGED>
__device__ __forceinline__ float4 update4(float L, const float4 &c, float R, const float4 &u, const float4 &d,
                                          float2 alpha2, float2 beta2, int rw)
{
    float rx = c.y, ry = c.z, rz = c.w;
    if (RAGGED) {
        rx = rw == 0 ? c.x : rx;
        ry = rw == 1 ? c.y : ry;
        rz = rw == 2 ? c.z : rz;
    }
    float2 h01 = make_float2(L + rx, c.x + ry);
    float2 h23 = make_float2(c.y + rz, c.z + R);
    float2 s01 = __fadd2_rn(h01, __fadd2_rn(make_float2(u.x, u.y), make_float2(d.x, d.y)));
    float2 s23 = __fadd2_rn(h23, __fadd2_rn(make_float2(u.z, u.w), make_float2(d.z, d.w)));
    float2 o01 = __ffma2_rn(alpha2, s01, __fmul2_rn(beta2, make_float2(c.x, c.y)));
    float2 o23 = __ffma2_rn(alpha2, s23, __fmul2_rn(beta2, make_float2(c.z, c.w)));
    return make_float4(o01.x, o01.y, o23.x, o23.y);
}

// Per-lane wall flags: the left x wall (global x = 0) falls on the first
// component of one of the lane's two float4 groups; the right wall (global
// x = nx - 1) on the last component (r_*) or, when nx % 4 != 0, inside a group
// (rw_* = 0..2; 4 = not in this group).
struct LaneWalls {
    bool l_a, r_a, l_b, r_b;
    int rw_a, rw_b;
};

__device__ __forceinline__ LaneWalls lane_walls(int gxA, int gxB, int nx)
{
    const int ea = nx - 1 - gxA, eb = nx - 1 - gxB;
    return LaneWalls{gxA == 0, ea == 3, gxB == 0, eb == 3, (ea >= 0 && ea < 3) ? ea : 4,
                     (eb >= 0 && eb < 3) ? eb : 4};
}

// New values of row `cur` from the old rows above/at/below.  x neighbours come
// from adjacent lanes.  The tile's two outermost columns take whatever the
// shuffle wraps around (they are outside the valid region after the first
// sub-step anyway); a node on an x wall uses itself as its missing neighbour.
template <bool RAGGED>
__device__ __forceinline__ Row update_row(const Row &up, const Row &cur, const Row &dn, int lane,
                                          const LaneWalls &w, float2 alpha2, float2 beta2)
{
    float aL = __shfl_sync(kFull, cur.a.w, (lane + 31) & 31);
    float aR = __shfl_sync(kFull, lane == 0 ? cur.b.x : cur.a.x, (lane + 1) & 31);
    float bL = __shfl_sync(kFull, lane == 31 ? cur.a.w : cur.b.w, (lane + 31) & 31);
    float bR = __shfl_sync(kFull, cur.b.x, (lane + 1) & 31);
    aL = w.l_a ? cur.a.x : aL;
    aR = w.r_a ? cur.a.w : aR;
    bL = w.l_b ? cur.b.x : bL;
    bR = w.r_b ? cur.b.w : bR;
    Row o;
    o.a = update4<RAGGED>(aL, cur.a, aR, up.a, dn.a, alpha2, beta2, w.rw_a);
    o.b = update4<RAGGED>(bL, cur.b, bR, up.b, dn.b, alpha2, beta2, w.rw_b);
    return o;
}

__device__ __forceinline__ float comp(const float4 &v, int k)
{
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

__device__ __forceinline__ void set_comp(float4 &v, int k, float e)
{
    if (k == 0) v.x = e;
    else if (k == 1) v.y = e;
    else if (k == 2) v.z = e;
    else v.w = e;
}

// Sources of one warp band, consumed in row order.
struct BandSources {
    const int *t_col, *t_row;
    const float *t_e;
    int begin, end;
};

// Dense rate map of the tile (MAP only): row r of the tile is global row
// oy + r; the lane's groups start at global columns gxA, gxB (reads only rows
// inside the grid and groups inside the row pitch).
struct BandMap {
    const float *map;
    int pitch, oy, ny, gxA, gxB;
    float dt;
};

__device__ __forceinline__ float4 fma4(float a, const float4 &m, const float4 &o)
{
    return make_float4(fmaf(a, m.x, o.x), fmaf(a, m.y, o.y), fmaf(a, m.z, o.z), fmaf(a, m.w, o.w));
}

// One sub-step of the in-place sweep over the warp's band of kBand rows
// starting at r0.  `above` / `below` are the old rows just outside the band,
// read before the CTA barrier that precedes the sweep.  On WALL tiles (a y
// wall inside the loaded rows), rows outside the domain are not stored and the
// ghost row beyond each y wall is rewritten with the new edge row, so the
// next sub-step sees the edge node as its own missing neighbour.  MAP adds
// dt M to every row inside the grid after the stencil, before the sources
// (the plain kernels' order).
template <bool WALL, bool RAGGED, bool MAP>
__device__ __forceinline__ void sweep_band(float4 *S4, int lane, int r0, const Row &above, const Row &below,
                                           const LaneWalls &lw, float2 alpha2, float2 beta2,
                                           const BandSources &src, int oy, int ny, const BandMap &bm)
{
    int sp = src.begin;
    int srow = sp < src.end ? src.t_row[sp] : 1 << 30;
    Row up = above;
    Row cur = ld_row(S4, r0, lane);
    Row dn = ld_row(S4, r0 + 1, lane);
#pragma unroll
    for (int i = 0; i < kBand; ++i) {
        const int r = r0 + i;
        Row nxt;
        if (i + 2 < kBand) nxt = ld_row(S4, r + 2, lane);
        else if (i + 2 == kBand) nxt = below;
        Row o = update_row<RAGGED>(up, cur, dn, lane, lw, alpha2, beta2);
        if (MAP) {
            const int gy = bm.oy + r;
            if (gy >= 0 && gy < bm.ny) {
                const float4 *mrow = reinterpret_cast<const float4 *>(bm.map + (size_t)gy * bm.pitch);
                if (bm.gxA >= 0 && bm.gxA < bm.pitch) o.a = fma4(bm.dt, __ldg(mrow + (bm.gxA >> 2)), o.a);
                if (bm.gxB >= 0 && bm.gxB < bm.pitch) o.b = fma4(bm.dt, __ldg(mrow + (bm.gxB >> 2)), o.b);
            }
        }
        while (srow == r) {
            const int col = src.t_col[sp];
            const float e = src.t_e[sp];
            const int q = col >> 2;
            if ((q & 31) == lane) {
                if (q < 32) set_comp(o.a, col & 3, comp(o.a, col & 3) + e);
                else set_comp(o.b, col & 3, comp(o.b, col & 3) + e);
            }
            ++sp;
            srow = sp < src.end ? src.t_row[sp] : 1 << 30;
        }
        if (WALL) {
            const int gy = oy + r;
            if (gy >= 0 && gy < ny) st_row(S4, r, lane, o);
            if (gy == 0 && r > 0) st_row(S4, r - 1, lane, o);               // top ghost row
            if (gy == ny - 1 && r + 1 < kRows) st_row(S4, r + 1, lane, o);  // bottom ghost row
        } else {
            st_row(S4, r, lane, o);
        }
        up = cur;
        cur = dn;
        dn = nxt;
    }
}

}  // namespace tile
}  // namespace cue
