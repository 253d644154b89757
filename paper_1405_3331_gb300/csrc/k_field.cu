// k_field.cu -- one explicit field step (rows a1, a2): the no-flux
// neighbour-difference stencil with decay, the optional dense rate map, and
// point-source emission.  These are the unfused kernels: one HBM/L2 round
// trip per step (8 B per node update, 12 B with a rate map).
//
// Update (Sec. 5.2 Eulerian grid, Sec. 4.3 sources with their own rates):
//   C'_i = C_i + alpha * sum_{existing axis nbrs j} (C_j - C_i) - decay * C_i
//          [+ dt * M_i] [+ e_k at source nodes]
// evaluated as beta C_i + alpha sum_j C_j with a missing neighbour (wall)
// replaced by the node itself (node_update2/3).
#include "cue_internal.h"

namespace cue {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool finite4(const float4 &v)
{
    const float big = 3.402823466e38f;
    return fabsf(v.x) <= big && fabsf(v.y) <= big && fabsf(v.z) <= big && fabsf(v.w) <= big;
}

// ---------------------------------------------------------------- 2D, float4
// Block = 32 lanes (x, 4 nodes each) x BY warps (y segments of `rows` rows).
// Each thread streams its 4-wide column strip down its rows, keeping the
// rows above/at/below in registers; x neighbours come from the adjacent lane
// by shuffle, and from global memory at the warp edges.
//
// Point sources are added by the block that owns their node, after the
// update of that node and in source order (the same rounding as a separate
// pass): the block first lists the sources inside its rectangle in shared
// memory, so a block without sources pays one pass over the source table.
constexpr int kBlockSources = 64;

template <bool MAP>
__global__ void __launch_bounds__(256) field2d_vec4(FieldDesc f, const float *__restrict__ Cin,
                                                    float *__restrict__ Cout,
                                                    const float *__restrict__ M, int rows,
                                                    const int32_t *__restrict__ src_cell,
                                                    const float *__restrict__ src_emit, int n_src,
                                                    unsigned *status)
{
    __shared__ int s_n;
    __shared__ int s_cell[kBlockSources];
    __shared__ float s_emit[kBlockSources];
    const int lane = threadIdx.x;
    const int nx4 = f.nx >> 2;
    const int x4 = blockIdx.x * 32 + lane;
    const bool xin = x4 < nx4;
    const int bx0 = blockIdx.x * 128, bx1 = min(bx0 + 128, f.nx);
    const int by0 = blockIdx.y * blockDim.y * rows, by1 = min(by0 + (int)blockDim.y * rows, f.ny);
    const int tid = threadIdx.y * 32 + lane;
    if (tid == 0) s_n = 0;
    __syncthreads();
    for (int k = tid; k < n_src; k += blockDim.x * blockDim.y) {
        const int c = src_cell[k];
        if (c < 0 || (long long)c >= (long long)f.nx * f.ny) {
            if (blockIdx.x == 0 && blockIdx.y == 0) flag_status(status, kStatusBounds);
            continue;
        }
        const int cx = c % f.nx, cy = c / f.nx;
        if (cx >= bx0 && cx < bx1 && cy >= by0 && cy < by1) {
            const int slot = atomicAdd(&s_n, 1);
            if (slot < kBlockSources) {
                s_cell[slot] = k;          // source index first: sorted below
            } else {
                flag_status(status, kStatusBounds);
            }
        }
    }
    __syncthreads();
    const int nb = min(s_n, kBlockSources);
    if (tid == 0 && nb > 1) {          // keep the table's order (ties add as a separate pass would)
        for (int i = 1; i < nb; ++i)
            for (int j = i; j > 0 && s_cell[j - 1] > s_cell[j]; --j) {
                const int t = s_cell[j];
                s_cell[j] = s_cell[j - 1];
                s_cell[j - 1] = t;
            }
    }
    __syncthreads();
    if (tid < nb) {
        const int k = s_cell[tid];
        s_emit[tid] = src_emit[k];
        s_cell[tid] = src_cell[k];
    }
    __syncthreads();
    const int y0 = (blockIdx.y * blockDim.y + threadIdx.y) * rows;
    if (y0 >= f.ny) return;                       // warp-uniform
    const int y1 = min(y0 + rows, f.ny);
    const int x = x4 * 4;
    const bool has_l = x > 0, has_r = x + 4 < f.nx;
    const float4 *in4 = reinterpret_cast<const float4 *>(Cin);
    float4 *out4 = reinterpret_cast<float4 *>(Cout);
    const float4 *m4 = reinterpret_cast<const float4 *>(M);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);

    float4 cur = xin ? __ldg(in4 + (size_t)y0 * nx4 + x4) : z4;
    float4 up = (xin && y0 > 0) ? __ldg(in4 + (size_t)(y0 - 1) * nx4 + x4) : cur;
    bool bad = false;
    for (int y = y0; y < y1; ++y) {
        float4 dn = (xin && y + 1 < f.ny) ? __ldg(in4 + (size_t)(y + 1) * nx4 + x4) : cur;
        float l = __shfl_up_sync(kFull, cur.w, 1);
        float r = __shfl_down_sync(kFull, cur.x, 1);
        if (lane == 0) l = (xin && has_l) ? __ldg(Cin + (size_t)y * f.nx + x - 1) : cur.x;
        if (lane == 31) r = (xin && has_r) ? __ldg(Cin + (size_t)y * f.nx + x + 4) : cur.w;
        if (!has_l) l = cur.x;
        if (!has_r) r = cur.w;
        if (xin) {
            float4 o;
            o.x = node_update2(cur.x, l, cur.y, up.x, dn.x, f.alpha, f.beta);
            o.y = node_update2(cur.y, cur.x, cur.z, up.y, dn.y, f.alpha, f.beta);
            o.z = node_update2(cur.z, cur.y, cur.w, up.z, dn.z, f.alpha, f.beta);
            o.w = node_update2(cur.w, cur.z, r, up.w, dn.w, f.alpha, f.beta);
            if constexpr (MAP) {
                float4 m = __ldg(m4 + (size_t)y * nx4 + x4);
                o.x = fmaf(f.dt, m.x, o.x);
                o.y = fmaf(f.dt, m.y, o.y);
                o.z = fmaf(f.dt, m.z, o.z);
                o.w = fmaf(f.dt, m.w, o.w);
            }
            for (int i = 0; i < nb; ++i) {
                const int c = s_cell[i] - y * f.nx - x;
                if (c == 0) o.x += s_emit[i];
                else if (c == 1) o.y += s_emit[i];
                else if (c == 2) o.z += s_emit[i];
                else if (c == 3) o.w += s_emit[i];
            }
            bad |= !finite4(o);
            out4[(size_t)y * nx4 + x4] = o;
        }
        up = cur;
        cur = dn;
    }
    if (__any_sync(kFull, bad) && lane == 0) flag_status(status, kStatusNonFinite);
}

// ---------------------------------------------------------------- 3D, float4
// Block = 32 lanes (x, 4 nodes each) x BY rows (y); each thread streams a
// chunk of z planes keeping z-1, z, z+1 in registers.  y neighbours come from
// a shared-memory copy of the block's plane row set (+1 halo row each side).
template <bool MAP, int BY>
__global__ void __launch_bounds__(32 * BY) field3d_vec4(FieldDesc f, const float *__restrict__ Cin,
                                                         float *__restrict__ Cout,
                                                         const float *__restrict__ M, int zchunk,
                                                         unsigned *status)
{
    __shared__ float4 tile[BY + 2][32];
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int nx4 = f.nx >> 2;
    const int x4 = blockIdx.x * 32 + lane;
    const bool xin = x4 < nx4;
    const int y = blockIdx.y * BY + ty;
    const bool act = xin && y < f.ny;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, f.nz);
    const int x = x4 * 4;
    const bool has_l = x > 0, has_r = x + 4 < f.nx;
    const size_t plane4 = (size_t)f.ny * nx4;
    const float4 *in4 = reinterpret_cast<const float4 *>(Cin);
    float4 *out4 = reinterpret_cast<float4 *>(Cout);
    const float4 *m4 = reinterpret_cast<const float4 *>(M);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto at = [&](int yy, int zz) { return (size_t)zz * plane4 + (size_t)yy * nx4 + x4; };

    float4 cur = act ? __ldg(in4 + at(y, z0)) : z4;
    float4 below = (act && z0 > 0) ? __ldg(in4 + at(y, z0 - 1)) : cur;
    bool bad = false;
    for (int z = z0; z < z1; ++z) {
        float4 above = (act && z + 1 < f.nz) ? __ldg(in4 + at(y, z + 1)) : cur;
        tile[ty + 1][lane] = cur;
        if (ty == 0) tile[0][lane] = (xin && y > 0) ? __ldg(in4 + at(y - 1, z)) : z4;
        if (ty == BY - 1) tile[BY + 1][lane] = (xin && y + 1 < f.ny) ? __ldg(in4 + at(y + 1, z)) : z4;
        __syncthreads();
        float4 s = (y > 0) ? tile[ty][lane] : cur;
        float4 n = (y + 1 < f.ny) ? tile[ty + 2][lane] : cur;
        float l = __shfl_up_sync(kFull, cur.w, 1);
        float r = __shfl_down_sync(kFull, cur.x, 1);
        const size_t row = (size_t)z * f.ny * f.nx + (size_t)y * f.nx;
        if (lane == 0) l = (act && has_l) ? __ldg(Cin + row + x - 1) : cur.x;
        if (lane == 31) r = (act && has_r) ? __ldg(Cin + row + x + 4) : cur.w;
        if (!has_l) l = cur.x;
        if (!has_r) r = cur.w;
        if (act) {
            float4 o;
            o.x = node_update3(cur.x, l, cur.y, s.x, n.x, below.x, above.x, f.alpha, f.beta);
            o.y = node_update3(cur.y, cur.x, cur.z, s.y, n.y, below.y, above.y, f.alpha, f.beta);
            o.z = node_update3(cur.z, cur.y, cur.w, s.z, n.z, below.z, above.z, f.alpha, f.beta);
            o.w = node_update3(cur.w, cur.z, r, s.w, n.w, below.w, above.w, f.alpha, f.beta);
            if constexpr (MAP) {
                float4 m = __ldg(m4 + at(y, z));
                o.x = fmaf(f.dt, m.x, o.x);
                o.y = fmaf(f.dt, m.y, o.y);
                o.z = fmaf(f.dt, m.z, o.z);
                o.w = fmaf(f.dt, m.w, o.w);
            }
            bad |= !finite4(o);
            out4[at(y, z)] = o;
        }
        __syncthreads();
        below = cur;
        cur = above;
    }
    if (__any_sync(kFull, bad) && lane == 0) flag_status(status, kStatusNonFinite);
}

// ---------------------------------------------------------------- any size
// One thread per node; used when nx is not a multiple of 4 or a buffer is not
// 16-byte aligned.
template <bool MAP>
__global__ void __launch_bounds__(256) field_scalar(FieldDesc f, const float *__restrict__ Cin,
                                                    float *__restrict__ Cout,
                                                    const float *__restrict__ M, unsigned *status)
{
    const size_t n = (size_t)f.nx * f.ny * f.nz;
    const size_t sy = f.nx, sz = (size_t)f.nx * f.ny;
    bool bad = false;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % f.nx);
        const int j = (int)((c / f.nx) % f.ny);
        const int k = (int)(c / sz);
        const float ci = __ldg(Cin + c);
        const float xm = i > 0 ? __ldg(Cin + c - 1) : ci;
        const float xp = i < f.nx - 1 ? __ldg(Cin + c + 1) : ci;
        const float ym = j > 0 ? __ldg(Cin + c - sy) : ci;
        const float yp = j < f.ny - 1 ? __ldg(Cin + c + sy) : ci;
        float o;
        if (f.dim == 3) {
            const float zm = k > 0 ? __ldg(Cin + c - sz) : ci;
            const float zp = k < f.nz - 1 ? __ldg(Cin + c + sz) : ci;
            o = node_update3(ci, xm, xp, ym, yp, zm, zp, f.alpha, f.beta);
        } else {
            o = node_update2(ci, xm, xp, ym, yp, f.alpha, f.beta);
        }
        if constexpr (MAP) o = fmaf(f.dt, __ldg(M + c), o);
        bad |= !(fabsf(o) <= 3.402823466e38f);
        Cout[c] = o;
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) flag_status(status, kStatusNonFinite);
}

// Point sources: C'[cell_k] += e_k (atomic, so duplicate cells accumulate).
__global__ void add_sources(float *C, size_t n_cells, const int32_t *__restrict__ cell,
                            const float *__restrict__ emit, int n_src, unsigned *status)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_src) return;
    int c = cell[s];
    if (c < 0 || (size_t)c >= n_cells) {
        flag_status(status, kStatusBounds);
        return;
    }
    atomicAdd(C + c, emit[s]);
}

// Source node coordinates [3][n_src] for the cones' squared-distance stop test.
__global__ void source_coords(FieldDesc f, const int32_t *__restrict__ cell, int n_src,
                              float *xyz, unsigned *status)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_src) return;
    long long c = cell[s];
    long long n = (long long)f.nx * f.ny * f.nz;
    if (c < 0 || c >= n) {
        flag_status(status, kStatusBounds);     // far away: never triggers the stop test
        xyz[s] = xyz[n_src + s] = xyz[2 * n_src + s] = 3.0e38f;
        return;
    }
    xyz[s] = (float)(c % f.nx) * f.h;
    xyz[n_src + s] = (float)((c / f.nx) % f.ny) * f.h;
    xyz[2 * n_src + s] = (float)(c / ((long long)f.nx * f.ny)) * f.h;
}

int sm_count()
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

cudaError_t launch_field_step(Sim &s, const float *Cin, float *Cout, bool *sources_done)
{
    const FieldDesc &f = s.fd;
    const bool map = s.src_map != nullptr;
    if (sources_done) *sources_done = false;
    timing_begin(s);
    if (s.vec4 && f.dim == 2) {
        const int nx4 = f.nx / 4;
        const int BY = 8;
        const int xb = (nx4 + 31) / 32;
        // rows per thread: the most register reuse that still leaves >= 4 blocks per SM
        int rows = s.rows_per_thread;
        if (rows <= 0) {
            rows = 8;
            while (rows > 1 && (long long)xb * ((f.ny + BY * rows - 1) / (BY * rows)) < 4LL * sm_count())
                rows /= 2;
        }
        dim3 grid(xb, (f.ny + BY * rows - 1) / (BY * rows));
        dim3 block(32, BY);
        const int ns = (sources_done && s.n_src <= kBlockSources) ? s.n_src : 0;
        if (map)
            field2d_vec4<true><<<grid, block, 0, s.stream>>>(f, Cin, Cout, s.src_map, rows, s.src_cell, s.src_emit,
                                                             ns, s.status());
        else
            field2d_vec4<false><<<grid, block, 0, s.stream>>>(f, Cin, Cout, nullptr, rows, s.src_cell, s.src_emit,
                                                              ns, s.status());
        if (sources_done) *sources_done = ns == s.n_src;
    } else if (s.vec4 && f.dim == 3 && (Cin == s.field[0] || Cin == s.field[1]) && field3d_tma_prepare(s)) {
        cudaError_t e = launch_field3d_tma(s, Cin == s.field[0] ? 0 : 1, Cout, nullptr, sources_done);
        timing_end(s);
        s.launches++;
        return e;
    } else if (s.vec4 && f.dim == 3) {
        constexpr int BY = 8;
        const int nx4 = f.nx / 4;
        const int xb = (nx4 + 31) / 32, yb = (f.ny + BY - 1) / BY;
        const long long target = 8LL * sm_count();
        int zchunk = f.nz;
        while (zchunk > 8 && (long long)xb * yb * ((f.nz + zchunk - 1) / zchunk) < target) zchunk /= 2;
        dim3 grid(xb, yb, (f.nz + zchunk - 1) / zchunk);
        dim3 block(32, BY);
        if (map) field3d_vec4<true, BY><<<grid, block, 0, s.stream>>>(f, Cin, Cout, s.src_map, zchunk, s.status());
        else field3d_vec4<false, BY><<<grid, block, 0, s.stream>>>(f, Cin, Cout, nullptr, zchunk, s.status());
    } else {
        const size_t n = (size_t)f.nx * f.ny * f.nz;
        size_t blocks = (n + 255) / 256;
        if (blocks > (size_t)sm_count() * 64) blocks = (size_t)sm_count() * 64;
        if (map) field_scalar<true><<<(unsigned)blocks, 256, 0, s.stream>>>(f, Cin, Cout, s.src_map, s.status());
        else field_scalar<false><<<(unsigned)blocks, 256, 0, s.stream>>>(f, Cin, Cout, nullptr, s.status());
    }
    timing_end(s);
    s.launches++;
    return cudaGetLastError();
}

cudaError_t launch_field_and_sources(Sim &s, const float *Cin, float *Cout)
{
    bool done = false;
    cudaError_t e = launch_field_step(s, Cin, Cout, &done);
    if (e == cudaSuccess && !done) e = launch_sources(s, Cout);
    return e;
}

cudaError_t launch_sources(Sim &s, float *Cout)
{
    if (s.n_src == 0) return cudaSuccess;
    const size_t n = (size_t)s.fd.nx * s.fd.ny * s.fd.nz;
    add_sources<<<(s.n_src + 127) / 128, 128, 0, s.stream>>>(Cout, n, s.src_cell, s.src_emit, s.n_src,
                                                             s.status());
    s.launches++;
    return cudaGetLastError();
}

cudaError_t launch_src_xyz(Sim &s)
{
    if (s.n_src == 0) return cudaSuccess;
    source_coords<<<(s.n_src + 127) / 128, 128, 0, s.stream>>>(s.fd, s.src_cell, s.n_src, s.src_xyz(),
                                                               s.status());
    s.launches++;
    return cudaGetLastError();
}

}  // namespace cue
