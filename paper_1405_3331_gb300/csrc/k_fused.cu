// k_fused.cu -- the fused, temporally blocked 2D path: one launch advances the
// field AND the growth cones K steps (rows a1-a6) with one HBM/L2 round trip
// of the field.
//
// Each CTA owns an interior tile of TX x TY nodes.  It loads the tile plus a
// halo (HX columns, HY rows on each side) into shared memory with one TMA
// tensor copy, then runs K sub-steps entirely in shared memory:
//   phase A  the cones binned to this tile take step n+j, reading C^{n+j}
//            from shared memory (multilinear gradient, Philox noise, blend,
//            advance, stop tests), state read from / written to global;
//   phase B  the field advances in place to C^{n+j+1}: each warp sweeps a
//            band of full-width rows, keeping the rows above/at/below in
//            registers (x neighbours by warp shuffle) and adding the point
//            sources of each row as it goes.
// After K sub-steps the interior is stored.  The valid region shrinks by one
// node per sub-step; cones move at most step_len per step and read a 4-node
// footprint, so the halo is H = K + 1 + ceil((K-1) step_len / h) (the x halo
// rounded up to 4 nodes for 16-byte TMA coordinates).  Cones are re-binned to
// tiles between launches (count, scan, scatter).
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

namespace cue {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kW = 256;               // loaded columns per tile: a warp spans a row, 2 float4 per lane
constexpr int kThreads = 256;         // 8 warps
constexpr int kWarps = kThreads / 32;
constexpr int kMaxTileSrc = 256;      // sources per tile (and in total on this path)
constexpr long long kWaitLimit = 1LL << 22;

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

// New values of row `cur` from the old rows above/at/below.  x neighbours come
// from adjacent lanes; the tile's outer columns (invalid rim) use the node
// itself; the walls (global x = 0 and x = nx-1) use the node itself.
__device__ __forceinline__ Row update_row(const Row &up, const Row &cur, const Row &dn, int lane,
                                          bool wl_a, bool wr_a, bool wl_b, bool wr_b, float alpha, float beta)
{
    float aL = __shfl_sync(kFull, cur.a.w, (lane + 31) & 31);
    float aR = __shfl_sync(kFull, lane == 0 ? cur.b.x : cur.a.x, (lane + 1) & 31);
    float bL = __shfl_sync(kFull, lane == 31 ? cur.a.w : cur.b.w, (lane + 31) & 31);
    float bR = __shfl_sync(kFull, cur.b.x, (lane + 1) & 31);
    if (lane == 0 || wl_a) aL = cur.a.x;
    if (wr_a) aR = cur.a.w;
    if (wl_b) bL = cur.b.x;
    if (lane == 31 || wr_b) bR = cur.b.w;
    Row o;
    o.a.x = node_update2(cur.a.x, aL, cur.a.y, up.a.x, dn.a.x, alpha, beta);
    o.a.y = node_update2(cur.a.y, cur.a.x, cur.a.z, up.a.y, dn.a.y, alpha, beta);
    o.a.z = node_update2(cur.a.z, cur.a.y, cur.a.w, up.a.z, dn.a.z, alpha, beta);
    o.a.w = node_update2(cur.a.w, cur.a.z, aR, up.a.w, dn.a.w, alpha, beta);
    o.b.x = node_update2(cur.b.x, bL, cur.b.y, up.b.x, dn.b.x, alpha, beta);
    o.b.y = node_update2(cur.b.y, cur.b.x, cur.b.z, up.b.y, dn.b.y, alpha, beta);
    o.b.z = node_update2(cur.b.z, cur.b.y, cur.b.w, up.b.z, dn.b.z, alpha, beta);
    o.b.w = node_update2(cur.b.w, cur.b.z, bR, up.b.w, dn.b.w, alpha, beta);
    return o;
}

__device__ __forceinline__ void add_comp(float4 &v, int k, float e)
{
    if (k == 0) v.x += e;
    else if (k == 1) v.y += e;
    else if (k == 2) v.z += e;
    else v.w += e;
}

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
    const int *bin_off, *bin_list;
    const int32_t *src_cell;
    const float *src_emit;
    int n_src;
    const float *src_xyz;
    unsigned *status;
    unsigned long long *counter;
};

__global__ void __launch_bounds__(kThreads, 2) fused2d_kernel(const __grid_constant__ CUtensorMap tmap,
                                                              const FusedArgs A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const FusedGeom &g = A.g;
    const FieldDesc &f = A.f;
    // layout: mbarrier at 0; the TMA tile at 128 (128-byte aligned); then the lists
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    float *S = reinterpret_cast<float *>(smem_raw + 128);
    float4 *S4 = reinterpret_cast<float4 *>(smem_raw + 128);
    int *row_start = reinterpret_cast<int *>(S + g.R * kW);    // R + 1
    int *row_fill = row_start + (g.R + 1);                      // R
    int *t_col = row_fill + g.R;                                // kMaxTileSrc
    float *t_e = reinterpret_cast<float *>(t_col + kMaxTileSrc);
    float *s_xy = t_e + kMaxTileSrc;                            // [2][kMaxTileSrc]

    const int t = blockIdx.x;
    const int tx = t % g.ntx, ty = t / g.ntx;
    const int ox = tx * g.TX - g.HX, oy = ty * g.TY - g.HY;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) mbar_init(bar, 1);
    for (int r = tid; r < g.R; r += kThreads) row_fill[r] = 0;
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(bar, (unsigned)(g.R * kW * sizeof(float)));
        tma_load_2d(S, &tmap, bar, ox, oy);
    }

    // point sources inside the loaded region, grouped by tile row (overlaps the TMA load)
    const bool stop_on = A.cones_on && A.c.stop_r2 >= 0.0f && A.n_src > 0;
    for (int s = tid; s < A.n_src; s += kThreads) {
        int cell = A.src_cell[s];
        if (cell >= 0 && cell < f.nx * f.ny) {
            int gx = cell % f.nx, gy = cell / f.nx;
            if (gx >= ox && gx < ox + kW && gy >= oy && gy < oy + g.R) atomicAdd(&row_fill[gy - oy], 1);
        }
        if (stop_on) {
            s_xy[s] = A.src_xyz[s];
            s_xy[kMaxTileSrc + s] = A.src_xyz[A.n_src + s];
        }
    }
    __syncthreads();
    if (warp == 0) {       // exclusive scan of the per-row counts
        int carry = 0;
        for (int base = 0; base < g.R; base += 32) {
            int r = base + lane;
            int v = r < g.R ? row_fill[r] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += y;
            }
            if (r < g.R) row_start[r] = carry + x - v;
            carry += __shfl_sync(kFull, x, 31);
        }
        if (lane == 0) row_start[g.R] = carry;
    }
    __syncthreads();
    for (int r = tid; r < g.R; r += kThreads) row_fill[r] = 0;
    __syncthreads();
    for (int s = tid; s < A.n_src; s += kThreads) {
        int cell = A.src_cell[s];
        if (cell >= 0 && cell < f.nx * f.ny) {
            int gx = cell % f.nx, gy = cell / f.nx;
            if (gx >= ox && gx < ox + kW && gy >= oy && gy < oy + g.R) {
                int r = gy - oy;
                int slot = row_start[r] + atomicAdd(&row_fill[r], 1);
                t_col[slot] = gx - ox;
                t_e[slot] = A.src_emit[s];
            }
        }
    }

    // wait for the tile (bounded)
    bool ok = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            flag_status(A.status, kStatusTimeout);
            mbar_wait_bounded(bar, 0);      // let an in-flight copy land before the CTA exits
        }
        return;
    }

    const int b0 = A.cones_on ? A.bin_off[t] : 0;
    const int b1 = A.cones_on ? A.bin_off[t + 1] : 0;
    const int r0 = warp * g.R / kWarps, r1 = (warp + 1) * g.R / kWarps;
    const int colA = 4 * lane, colB = 128 + 4 * lane;
    const int gxA = ox + colA, gxB = ox + colB;
    const bool wl_a = gxA == 0, wl_b = gxB == 0;
    const bool wr_a = gxA + 3 == f.nx - 1, wr_b = gxB + 3 == f.nx - 1;
    const int n = A.n_axons;

    auto ld = [&](int i, int j, int) {
        int lx = i - ox, ly = j - oy;
        if ((unsigned)lx >= (unsigned)kW || (unsigned)ly >= (unsigned)g.R) {
            flag_status(A.status, kStatusBounds);
            lx = min(max(lx, 0), kW - 1);
            ly = min(max(ly, 0), g.R - 1);
        }
        return S[ly * kW + lx];
    };

    for (int j = 0; j < A.K; ++j) {
        // ---- phase A: cones of this tile read C^{n+j}
        for (int base = b0; base < b1; base += kThreads) {
            int i = base + tid;
            int a = i < b1 ? A.bin_list[i] : -1;
            bool live = a >= 0 && A.active[a];
            count_active(A.counter, live);
            if (live) {
                float p[2] = {A.pos[a], A.pos[n + a]};
                float d[2] = {A.dir[a], A.dir[n + a]};
                bool alive = cone_update<2>(f, A.c, ld, (uint32_t)a, A.step0 + j, p, d, s_xy, kMaxTileSrc,
                                            stop_on ? A.n_src : 0);
                A.pos[a] = p[0];
                A.pos[n + a] = p[1];
                A.dir[a] = d[0];
                A.dir[n + a] = d[1];
                if (!alive) A.active[a] = 0;
            }
        }
        // rows just outside this warp's band, read before anyone overwrites them
        Row above, below;
        const bool has_above = r0 > 0, has_below = r1 < g.R;
        if (has_above) above = ld_row(S4, r0 - 1, lane);
        if (has_below) below = ld_row(S4, r1, lane);
        __syncthreads();
        // ---- phase B: in-place sweep of the band to C^{n+j+1}
        Row cur = ld_row(S4, r0, lane);
        Row up = has_above ? above : cur;
        for (int r = r0; r < r1; ++r) {
            Row dn = (r + 1 < r1) ? ld_row(S4, r + 1, lane) : (has_below ? below : cur);
            const int gy = oy + r;
            const Row &u2 = (gy == 0) ? cur : up;
            const Row &d2 = (gy == f.ny - 1) ? cur : dn;
            Row o = update_row(u2, cur, d2, lane, wl_a, wr_a, wl_b, wr_b, f.alpha, f.beta);
            for (int s = row_start[r], s1 = row_start[r + 1]; s < s1; ++s) {
                int col = t_col[s];
                float e = t_e[s];
                if ((col >> 2) == lane) add_comp(o.a, col & 3, e);
                else if (((col - 128) >> 2) == lane && col >= 128) add_comp(o.b, col & 3, e);
            }
            st_row(S4, r, lane, o);
            up = cur;
            cur = dn;
        }
        __syncthreads();
    }

    // ---- store the interior
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
__global__ void bin_count_kernel(FieldDesc f, FusedGeom g, int n, const float *__restrict__ pos,
                                 const uint8_t *__restrict__ active, int *count, int *cone_tile, int *cone_slot)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    if (!active[a]) {
        cone_tile[a] = -1;
        return;
    }
    int ix = clampi((int)floorf(pos[a] / f.h), 0, f.nx - 1);
    int iy = clampi((int)floorf(pos[n + a] / f.h), 0, f.ny - 1);
    int tile = (iy / g.TY) * g.ntx + ix / g.TX;
    cone_tile[a] = tile;
    cone_slot[a] = atomicAdd(&count[tile], 1);
}

// Every block scans the per-tile counts (exclusive) in shared memory, then
// scatters its cones into the bin list; block 0 publishes the offsets.  The
// counts of the next round are cleared here.
__global__ void __launch_bounds__(1024) bin_scatter_kernel(int n_tiles, int n, const int *__restrict__ count,
                                                           int *count_next, int *bin_off, int *bin_list,
                                                           const int *__restrict__ cone_tile,
                                                           const int *__restrict__ cone_slot)
{
    extern __shared__ int s_off[];     // n_tiles + 1
    __shared__ int s_part[1024 / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n_tiles + blockDim.x - 1) / blockDim.x;
    const int lo = min(tid * per, n_tiles), hi = min(lo + per, n_tiles);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += count[i];
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_part[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int v = lane < (int)(blockDim.x / 32) ? s_part[lane] : 0;
        int y = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int z = __shfl_up_sync(kFull, y, o);
            if (lane >= o) y += z;
        }
        if (lane < (int)(blockDim.x / 32)) s_part[lane] = y - v;
    }
    __syncthreads();
    int run = s_part[warp] + x - sum;
    for (int i = lo; i < hi; ++i) {
        s_off[i] = run;
        run += count[i];
    }
    if (tid == blockDim.x - 1) s_off[n_tiles] = run;
    __syncthreads();
    if (blockIdx.x == 0)
        for (int i = tid; i <= n_tiles; i += blockDim.x) bin_off[i] = s_off[i];
    for (int i = blockIdx.x * blockDim.x + tid; i < n_tiles; i += gridDim.x * blockDim.x) count_next[i] = 0;
    for (int a = blockIdx.x * blockDim.x + tid; a < n; a += gridDim.x * blockDim.x) {
        int tile = cone_tile[a];
        if (tile >= 0) bin_list[s_off[tile] + cone_slot[a]] = a;
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
    return 128 + (size_t)R * kW * sizeof(float) + sizeof(int) * (2 * R + 1) + sizeof(int) * kMaxTileSrc +
           sizeof(float) * 3 * kMaxTileSrc;
}

// Tile geometry for temporal depth K; returns false if the fused path cannot run.
bool choose_geometry(const FieldDesc &f, float step_len, bool cones, int K, int sms, FusedGeom &g)
{
    if (f.dim != 2 || K < 1 || K > kMaxTemporalDepth) return false;
    double drift = cones ? std::ceil((K - 1) * (double)step_len / (double)f.h * (1.0 + 1e-5)) : 0.0;
    int H = cones ? (int)(K + 1 + drift) : K;
    int HX = (H + 3) & ~3;
    if (kW - 2 * HX < 32) return false;
    const int candidates[2][2] = {{100, 2}, {208, 1}};   // rows, CTAs per SM
    double best = 1e300;
    bool found = false;
    for (auto &cand : candidates) {
        int R = cand[0], cps = cand[1];
        int TY = R - 2 * H;
        if (TY < 8) continue;
        int TX = kW - 2 * HX;
        long long ntx = (f.nx + TX - 1) / TX, nty = (f.ny + TY - 1) / TY;
        long long tiles = ntx * nty;
        long long slots = (long long)sms * cps;
        double waves = (double)((tiles + slots - 1) / slots);
        double cost = waves * cps * R;
        if (cost < best) {
            best = cost;
            g.W = kW;
            g.R = R;
            g.HX = HX;
            g.HY = H;
            g.TX = TX;
            g.TY = TY;
            g.ntx = (int)ntx;
            g.nty = (int)nty;
            g.K = K;
            g.ctas_per_sm = cps;
            found = true;
        }
    }
    return found;
}

}  // namespace

// Upper bound on the tile count of any geometry (TX >= 32, TY >= 8), used to
// size the binning workspace independently of the temporal depth.
int fused_tile_count(const cue_params &p)
{
    if (p.dim != 2) return 0;
    long long n = (long long)((p.nx + 31) / 32) * ((p.ny + 7) / 8);
    return n > (1 << 22) ? 0 : (int)n;
}

static int default_depth(const Sim &s) { return s.temporal_depth > 0 ? s.temporal_depth : 8; }

bool fused_supported(const Sim &s)
{
    if (s.fd.dim != 2 || !s.vec4 || s.src_map || s.n_src > kMaxTileSrc) return false;
    if (!encode_fn()) return false;
    FusedGeom g;
    if (!choose_geometry(s.fd, s.cd.step_len, s.n_axons > 0, default_depth(s), device_sm_count(), g))
        return false;
    long long tiles = (long long)g.ntx * g.nty;
    if (tiles > s.wl.n_tiles || tiles + 1 > 16384) return false;
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
    if (!choose_geometry(s.fd, s.cd.step_len, s.n_axons > 0, K, device_sm_count(), g)) return CUE_ERR_ARG;
    s.geom = g;
    if (!make_maps(s)) return CUE_ERR_CUDA;
    size_t smem = fused_smem_bytes(g.R);
    if (cudaFuncSetAttribute(fused2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return CUE_ERR_CUDA;
    const int scan_smem = (int)(sizeof(int) * (g.ntx * g.nty + 1));
    if (scan_smem > 48 * 1024 &&
        cudaFuncSetAttribute(bin_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, scan_smem) !=
            cudaSuccess)
        return CUE_ERR_CUDA;
    s.geom_ready = true;
    return CUE_OK;
}

// One launch of k <= K fused steps (cones on or off) from s.cur into s.cur^1.
static cudaError_t launch_fused(Sim &s, int k, bool cones)
{
    const FusedGeom &g = s.geom;
    const int n_tiles = g.ntx * g.nty;
    int *count = s.bin_count();
    int *cur_count = count + (s.bin_round & 1) * s.wl.n_tiles;
    int *next_count = count + ((s.bin_round + 1) & 1) * s.wl.n_tiles;
    if (cones && s.n_axons > 0) {
        bin_count_kernel<<<(s.n_axons + 255) / 256, 256, 0, s.stream>>>(s.fd, g, s.n_axons, s.pos, s.active, cur_count,
                                                                         s.cone_tile(), s.cone_slot());
        s.launches++;
        int blocks = (s.n_axons + 1023) / 1024;
        size_t sm = sizeof(int) * (n_tiles + 1);
        bin_scatter_kernel<<<blocks, 1024, sm, s.stream>>>(n_tiles, s.n_axons, cur_count, next_count, s.bin_off(),
                                                           s.bin_list(), s.cone_tile(), s.cone_slot());
        s.launches++;
        s.bin_round++;
    }
    FusedArgs A;
    A.f = s.fd;
    A.c = s.cd;
    A.g = g;
    A.Cout = s.field[s.cur ^ 1];
    A.K = k;
    A.step0 = (uint32_t)s.field_step;
    A.cones_on = (cones && s.n_axons > 0) ? 1 : 0;
    A.n_axons = s.n_axons;
    A.pos = s.pos;
    A.dir = s.dir;
    A.active = s.active;
    A.bin_off = s.bin_off();
    A.bin_list = s.bin_list();
    A.src_cell = s.src_cell;
    A.src_emit = s.src_emit;
    A.n_src = s.n_src;
    A.src_xyz = s.src_xyz();
    A.status = s.status();
    A.counter = s.cone_counter();
    const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(s.tmap[s.cur]);
    timing_begin(s);
    fused2d_kernel<<<n_tiles, kThreads, fused_smem_bytes(g.R), s.stream>>>(*map, A);
    timing_end(s);
    s.launches++;
    return cudaGetLastError();
}

int run_fused_if_supported(Sim &s, int nsteps)
{
    if (s.path == CUE_PATH_PLAIN) return 1;
    if (!fused_supported(s)) {
        if (s.path == CUE_PATH_FUSED) return CUE_ERR_ARG;
        return 1;
    }
    int rc = prepare(s);
    if (rc != CUE_OK) return s.path == CUE_PATH_FUSED ? rc : 1;
    while (nsteps > 0) {
        int k = nsteps < s.geom.K ? nsteps : s.geom.K;
        if (launch_fused(s, k, true) != cudaSuccess) return CUE_ERR_CUDA;
        s.cur ^= 1;
        s.field_step += k;
        s.cone_step += k;
        nsteps -= k;
    }
    s.fused_used = true;
    return CUE_OK;
}

int field_fused_if_supported(Sim &s, int nsteps)
{
    if (s.path == CUE_PATH_PLAIN) return 1;
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
