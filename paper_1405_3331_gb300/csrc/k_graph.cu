// k_graph.cu -- the connectivity stage (include/cue_graph.h): uniform-grid
// binning (hash, sort, cell start; Sec. 3.5, Table 1), growth-cone / neuron
// connections (squared distances; Sec. 3.3), the adjacency list (Fig. 4) and
// level-synchronous breadth-first search (Fig. 5).
//
// The sort is a counting sort: cell counts (atomics), an exclusive scan, a
// scatter, then each cell's ids put in order by one thread, so the result is
// the (cell, id) order whatever order the atomics ran in.  Cell and distance
// decisions are taken in FP64 (a few operations per point or candidate pair),
// the precision of the definition they implement.
#include <algorithm>

#include "cue_barrier.cuh"
#include "cue_graph.h"
#include "cue_internal.h"

namespace cue {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanBlock = 1024;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
int blocks_of(long long n, int per) { return (int)((n + per - 1) / per); }

// ---------------------------------------------------------------- exclusive scan
// Block-wise scan of 1024 entries (warp shuffles, then the warp totals), the
// block totals scanned by one block with a running carry, then added back.
__device__ __forceinline__ int block_inclusive(int x, int *warp_tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    const int r = x + (w > 0 ? warp_tot[w - 1] : 0);
    __syncthreads();                                     // warp_tot is reused by the next call
    return r;
}

__global__ void __launch_bounds__(kScanBlock) scan_blocks(const int *in, int *out, int n, int *sums)
{
    __shared__ int warp_tot[32];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    const int incl = block_inclusive(v, warp_tot);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(kScanBlock) scan_sums(int *sums, int nb)
{
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += kScanBlock) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? sums[i] : 0;
        const int incl = block_inclusive(v, warp_tot);
        const int c = carry;
        if (i < nb) sums[i] = c + incl - v;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry = c + incl;
        __syncthreads();
    }
}

__global__ void scan_add(int *out, int n, const int *sums)
{
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
}

size_t scan_ws(long long n) { return al256(sizeof(int) * (size_t)std::max(1, blocks_of(n, kScanBlock))); }

cudaError_t exclusive_scan(const int *in, int *out, int n, int *sums, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int nb = blocks_of(n, kScanBlock);
    scan_blocks<<<nb, kScanBlock, 0, st>>>(in, out, n, sums);
    scan_sums<<<1, kScanBlock, 0, st>>>(sums, nb);
    scan_add<<<nb, kScanBlock, 0, st>>>(out, n, sums);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- binning
struct Grid3 {
    int dim, g[3];
    double cell;
};

__device__ __forceinline__ int axis_cell(double x, const Grid3 &G, int ax)
{
    long long k = (long long)floor(x / G.cell);
    k = k < 0 ? 0 : k;
    k = k > G.g[ax] - 1 ? G.g[ax] - 1 : k;
    return (int)k;
}

__global__ void bin_hash(Grid3 G, int n, const float *__restrict__ pos, int *cell_of, int *count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long c = 0, stride = 1;
    for (int ax = 0; ax < G.dim; ++ax) {
        c += (long long)axis_cell((double)pos[(size_t)ax * n + i], G, ax) * stride;
        stride *= G.g[ax];
    }
    cell_of[i] = (int)c;
    atomicAdd(count + c, 1);
}

__global__ void bin_scatter(int n, const int *__restrict__ cell_of, const int *__restrict__ start, int *cursor,
                            int *sorted_id, int *sorted_cell)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell_of[i];
    const int slot = start[c] + atomicAdd(cursor + c, 1);
    sorted_id[slot] = i;
    sorted_cell[slot] = c;
}

// Each cell's ids in ascending order (insertion sort by the cell's thread).
__global__ void sort_segments(int nseg, const int *__restrict__ start, const int *__restrict__ count, int *ids)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nseg) return;
    const int b = start[c], k = count[c];
    for (int i = b + 1; i < b + k; ++i) {
        const int v = ids[i];
        int j = i - 1;
        while (j >= b && ids[j] > v) {
            ids[j + 1] = ids[j];
            --j;
        }
        ids[j + 1] = v;
    }
}

// The paper's identifyCellStart: one thread per sorted entry; where the cell id
// differs from the previous (next) entry's, this entry starts (ends) its cell.
__global__ void identify_cell_start(int n, const int *__restrict__ sorted_cell, int *cell_start, int *cell_end)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int c = sorted_cell[j];
    if (j == 0 || sorted_cell[j - 1] != c) cell_start[c] = j;
    if (j == n - 1 || sorted_cell[j + 1] != c) cell_end[c] = j + 1;
}

struct BinLayout {
    size_t count, start, cursor, sorted_cell, sums, total;
};

BinLayout bin_layout(int n, long long ncell)
{
    BinLayout L{};
    size_t off = 0;
    L.count = off;
    off += al256(sizeof(int) * (size_t)ncell);
    L.start = off;
    off += al256(sizeof(int) * (size_t)ncell);
    L.cursor = off;
    off += al256(sizeof(int) * (size_t)ncell);
    L.sorted_cell = off;
    off += al256(sizeof(int) * (size_t)std::max(n, 1));
    L.sums = off;
    off += scan_ws(ncell);
    L.total = off;
    return L;
}

bool grid_ok(int dim, const int32_t *grid, long long *ncell)
{
    if ((dim != 2 && dim != 3) || !grid) return false;
    long long nc = 1;
    for (int ax = 0; ax < dim; ++ax) {
        if (grid[ax] < 1) return false;
        nc *= grid[ax];
        if (nc > (1LL << 30)) return false;
    }
    *ncell = nc;
    return true;
}

Grid3 make_grid(int dim, const int32_t *grid, float cell)
{
    Grid3 G{};
    G.dim = dim;
    G.g[0] = grid[0];
    G.g[1] = grid[1];
    G.g[2] = dim == 3 ? grid[2] : 1;
    G.cell = cell;
    return G;
}

// ---------------------------------------------------------------- connections
__global__ void connect_kernel(Grid3 G, int n_cones, const float *__restrict__ pos, const int *__restrict__ owner,
                               const uint8_t *__restrict__ active, int n_neurons, const float *__restrict__ npos,
                               double r2, const int *__restrict__ sorted_id, const int *__restrict__ cell_start,
                               const int *__restrict__ cell_end, int cap, int *src, int *dst, int *count)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_cones || (active && !active[a])) return;
    double x[3] = {0.0, 0.0, 0.0};
    int k[3] = {0, 0, 0};
    for (int ax = 0; ax < G.dim; ++ax) {
        x[ax] = (double)pos[(size_t)ax * n_cones + a];
        k[ax] = axis_cell(x[ax], G, ax);
    }
    const int me = owner[a];
    const int zr = G.dim == 3 ? 1 : 0;
    for (int dz = -zr; dz <= zr; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int cx = k[0] + dx, cy = k[1] + dy, cz = k[2] + dz;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= G.g[0] || cy >= G.g[1] || cz >= G.g[2]) continue;
                const long long c = cx + (long long)G.g[0] * (cy + (long long)G.g[1] * cz);
                const int b = cell_start[c];
                if (b < 0) continue;
                const int e = cell_end[c];
                for (int j = b; j < e; ++j) {
                    const int nid = sorted_id[j];
                    if (nid == me) continue;
                    double d2 = 0.0;
                    for (int ax = 0; ax < G.dim; ++ax) {
                        const double d = x[ax] - (double)npos[(size_t)ax * n_neurons + nid];
                        d2 += d * d;
                    }
                    if (d2 < r2) {
                        const int slot = atomicAdd(count, 1);
                        if (slot < cap) {
                            src[slot] = me;
                            dst[slot] = nid;
                        }
                    }
                }
            }
}

// ---------------------------------------------------------------- adjacency list
__global__ void csr_count(int nv, int ne_cap, const int *__restrict__ d_ne, const int *__restrict__ src,
                          const int *__restrict__ dst, int *deg)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int ne = min(*d_ne, ne_cap);
    if (k >= ne) return;
    const int s = src[k], d = dst[k];
    if (s < 0 || s >= nv || d < 0 || d >= nv) return;
    atomicAdd(deg + s, 1);
}

__global__ void csr_scatter(int nv, int ne_cap, const int *__restrict__ d_ne, const int *__restrict__ src,
                            const int *__restrict__ dst, const int *__restrict__ off, int *cursor, int *tmp)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int ne = min(*d_ne, ne_cap);
    if (k >= ne) return;
    const int s = src[k], d = dst[k];
    if (s < 0 || s >= nv || d < 0 || d >= nv) return;
    tmp[off[s] + atomicAdd(cursor + s, 1)] = d;
}

// Per vertex: its targets in order, duplicates dropped; uniq[v] their count.
__global__ void csr_dedupe(int nv, const int *__restrict__ off, const int *__restrict__ deg, int *tmp, int *uniq)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v > nv) return;
    if (v == nv) {
        uniq[nv] = 0;                                    // so the scan's last entry is the total
        return;
    }
    const int b = off[v], k = deg[v];
    for (int i = b + 1; i < b + k; ++i) {
        const int x = tmp[i];
        int j = i - 1;
        while (j >= b && tmp[j] > x) {
            tmp[j + 1] = tmp[j];
            --j;
        }
        tmp[j + 1] = x;
    }
    int m = 0;
    for (int i = b; i < b + k; ++i)
        if (i == b || tmp[i] != tmp[i - 1]) tmp[b + m++] = tmp[i];
    uniq[v] = m;
}

__global__ void csr_compact(int nv, const int *__restrict__ off, const int *__restrict__ uniq,
                            const int *__restrict__ row, const int *__restrict__ tmp, int *col, int *d_m)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v > nv) return;
    if (v == nv) {
        *d_m = row[nv];
        return;
    }
    for (int i = 0; i < uniq[v]; ++i) col[row[v] + i] = tmp[off[v] + i];
}

struct CsrLayout {
    size_t deg, off, cursor, tmp, uniq, sums, total;
};

CsrLayout csr_layout(int nv, int ne_cap)
{
    CsrLayout L{};
    size_t off = 0;
    L.deg = off;
    off += al256(sizeof(int) * (size_t)(nv + 1));
    L.off = off;
    off += al256(sizeof(int) * (size_t)(nv + 1));
    L.cursor = off;
    off += al256(sizeof(int) * (size_t)(nv + 1));
    L.tmp = off;
    off += al256(sizeof(int) * (size_t)std::max(ne_cap, 1));
    L.uniq = off;
    off += al256(sizeof(int) * (size_t)(nv + 1));
    L.sums = off;
    off += scan_ws(nv + 1);
    L.total = off;
    return L;
}

// ---------------------------------------------------------------- breadth-first search
// Fig. 5's arrays: F (frontier), X (visited, here level >= 0), C (cost =
// level).  Fig. 5 sets F[nid] in the same pass that reads F, so a vertex found
// at this level could be expanded within it; the levels stay exact here with
// two frontier arrays: level L expands the vertices of F[L % 2] and writes the
// vertices it finds into F[(L + 1) % 2], each claimed once by a compare-and-swap
// of its level from -1 to L + 1, then the grid meets at one barrier (the level
// synchronisation the text describes).  Three flag words rotate: level L sets
// flag[L % 3] when it finds a vertex and clears flag[(L + 1) % 3], last read
// after the barrier before the previous one.
__global__ void __launch_bounds__(256) bfs_kernel(int nv, const int *__restrict__ row, const int *__restrict__ col,
                                                  int source, int *level, uint8_t *F0, uint8_t *F1, int *flag,
                                                  PBar *bar, unsigned expected, long long limit, unsigned *status)
{
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int v = t0; v < nv; v += stride) {
        level[v] = v == source ? 0 : -1;
        F0[v] = v == source;
        F1[v] = 0;
    }
    if (!grid_barrier(bar, expected, limit, status)) return;
    for (int L = 0; L < nv; ++L) {
        uint8_t *Fc = (L & 1) ? F1 : F0, *Fn = (L & 1) ? F0 : F1;
        bool found = false;
        for (int v = t0; v < nv; v += stride) {
            if (!__ldcg(Fc + v)) continue;
            Fc[v] = 0;
            const int e1 = row[v + 1];
            for (int e = row[v]; e < e1; ++e) {
                const int u = col[e];
                if (__ldcg(level + u) < 0 && atomicCAS(level + u, -1, L + 1) == -1) {
                    Fn[u] = 1;
                    found = true;
                }
            }
        }
        if (t0 == 0) flag[(L + 1) % 3] = 0;
        if (__syncthreads_or(found) && threadIdx.x == 0) flag[L % 3] = 1;
        if (!grid_barrier(bar, expected, limit, status)) return;
        if (!__ldcg(flag + L % 3)) break;
    }
}

struct BfsLayout {
    size_t status, bar, flag, F, U, total;
};

BfsLayout bfs_layout(int nv)
{
    BfsLayout L{};
    L.status = 0;
    L.bar = 256;
    L.flag = 512;
    L.F = 768;
    L.U = L.F + al256((size_t)std::max(nv, 1));
    L.total = L.U + al256((size_t)std::max(nv, 1));
    return L;
}

int sm_count_g()
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

bool ws_ok(const void *ws, size_t have, size_t need)
{
    return ws && have >= need && (reinterpret_cast<uintptr_t>(ws) & 255u) == 0;
}

}  // namespace
}  // namespace cue

using namespace cue;

extern "C" {

size_t cue_bin_workspace_bytes(int32_t n, int64_t n_cells)
{
    if (n < 0 || n_cells <= 0 || n_cells > (1LL << 30)) return 0;
    return bin_layout(n, n_cells).total;
}

int cue_bin_points(int32_t dim, int32_t n, const float *d_pos, float cell, const int32_t *grid, int32_t *d_cell_of,
                   int32_t *d_sorted_id, int32_t *d_cell_start, int32_t *d_cell_end, void *d_ws, size_t ws_bytes,
                   void *stream)
{
    long long ncell = 0;
    if (!grid_ok(dim, grid, &ncell) || n < 0 || !(cell > 0.0f) || !std::isfinite(cell)) return CUE_ERR_ARG;
    if (n > 0 && (!d_pos || !d_cell_of || !d_sorted_id)) return CUE_ERR_ARG;
    if (!d_cell_start || !d_cell_end) return CUE_ERR_ARG;
    const BinLayout L = bin_layout(n, ncell);
    if (!ws_ok(d_ws, ws_bytes, L.total)) return CUE_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *W = static_cast<unsigned char *>(d_ws);
    int *count = reinterpret_cast<int *>(W + L.count), *start = reinterpret_cast<int *>(W + L.start);
    int *cursor = reinterpret_cast<int *>(W + L.cursor), *scell = reinterpret_cast<int *>(W + L.sorted_cell);
    int *sums = reinterpret_cast<int *>(W + L.sums);
    const Grid3 G = make_grid(dim, grid, cell);
    if (cudaMemsetAsync(count, 0, sizeof(int) * ncell, st) != cudaSuccess ||
        cudaMemsetAsync(cursor, 0, sizeof(int) * ncell, st) != cudaSuccess ||
        cudaMemsetAsync(d_cell_start, 0xFF, sizeof(int) * ncell, st) != cudaSuccess ||
        cudaMemsetAsync(d_cell_end, 0xFF, sizeof(int) * ncell, st) != cudaSuccess)
        return CUE_ERR_CUDA;
    if (n == 0) return CUE_OK;
    bin_hash<<<blocks_of(n, 256), 256, 0, st>>>(G, n, d_pos, d_cell_of, count);
    if (exclusive_scan(count, start, (int)ncell, sums, st) != cudaSuccess) return CUE_ERR_CUDA;
    bin_scatter<<<blocks_of(n, 256), 256, 0, st>>>(n, d_cell_of, start, cursor, d_sorted_id, scell);
    sort_segments<<<blocks_of(ncell, 256), 256, 0, st>>>((int)ncell, start, count, d_sorted_id);
    identify_cell_start<<<blocks_of(n, 256), 256, 0, st>>>(n, scell, d_cell_start, d_cell_end);
    return cudaGetLastError() == cudaSuccess ? CUE_OK : CUE_ERR_CUDA;
}

int cue_connect(int32_t dim, int32_t n_cones, const float *d_pos, const int32_t *d_owner, const uint8_t *d_active,
                int32_t n_neurons, const float *d_npos, float radius, float cell, const int32_t *grid,
                const int32_t *d_sorted_id, const int32_t *d_cell_start, const int32_t *d_cell_end, int32_t cap,
                int32_t *d_src, int32_t *d_dst, int32_t *d_count, void *stream)
{
    long long ncell = 0;
    if (!grid_ok(dim, grid, &ncell) || n_cones < 0 || n_neurons < 0 || cap < 0 || !d_count) return CUE_ERR_ARG;
    if (!(radius >= 0.0f) || !(cell >= radius) || !std::isfinite(cell) || !(cell > 0.0f)) return CUE_ERR_ARG;
    if (n_cones > 0 && (!d_pos || !d_owner)) return CUE_ERR_ARG;
    if (n_neurons > 0 && (!d_npos || !d_sorted_id || !d_cell_start || !d_cell_end)) return CUE_ERR_ARG;
    if (cap > 0 && (!d_src || !d_dst)) return CUE_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_count, 0, sizeof(int32_t), st) != cudaSuccess) return CUE_ERR_CUDA;
    if (n_cones == 0 || n_neurons == 0) return CUE_OK;
    const Grid3 G = make_grid(dim, grid, cell);
    connect_kernel<<<blocks_of(n_cones, 128), 128, 0, st>>>(G, n_cones, d_pos, d_owner, d_active, n_neurons, d_npos,
                                                            (double)radius * (double)radius, d_sorted_id,
                                                            d_cell_start, d_cell_end, cap, d_src, d_dst, d_count);
    return cudaGetLastError() == cudaSuccess ? CUE_OK : CUE_ERR_CUDA;
}

size_t cue_csr_workspace_bytes(int32_t nv, int32_t ne_cap)
{
    if (nv < 0 || ne_cap < 0 || nv >= (1 << 30)) return 0;
    return csr_layout(nv, ne_cap).total;
}

int cue_csr_build(int32_t nv, int32_t ne_cap, const int32_t *d_ne, const int32_t *d_src, const int32_t *d_dst,
                  int32_t *d_row, int32_t *d_col, int32_t *d_m, void *d_ws, size_t ws_bytes, void *stream)
{
    if (nv < 0 || nv >= (1 << 30) || ne_cap < 0 || !d_ne || !d_row || !d_m) return CUE_ERR_ARG;
    if (ne_cap > 0 && (!d_src || !d_dst || !d_col)) return CUE_ERR_ARG;
    const CsrLayout L = csr_layout(nv, ne_cap);
    if (!ws_ok(d_ws, ws_bytes, L.total)) return CUE_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *W = static_cast<unsigned char *>(d_ws);
    int *deg = reinterpret_cast<int *>(W + L.deg), *off = reinterpret_cast<int *>(W + L.off);
    int *cursor = reinterpret_cast<int *>(W + L.cursor), *tmp = reinterpret_cast<int *>(W + L.tmp);
    int *uniq = reinterpret_cast<int *>(W + L.uniq), *sums = reinterpret_cast<int *>(W + L.sums);
    if (cudaMemsetAsync(deg, 0, sizeof(int) * (nv + 1), st) != cudaSuccess ||
        cudaMemsetAsync(cursor, 0, sizeof(int) * (nv + 1), st) != cudaSuccess)
        return CUE_ERR_CUDA;
    if (ne_cap > 0) csr_count<<<blocks_of(ne_cap, 256), 256, 0, st>>>(nv, ne_cap, d_ne, d_src, d_dst, deg);
    if (exclusive_scan(deg, off, nv + 1, sums, st) != cudaSuccess) return CUE_ERR_CUDA;
    if (ne_cap > 0)
        csr_scatter<<<blocks_of(ne_cap, 256), 256, 0, st>>>(nv, ne_cap, d_ne, d_src, d_dst, off, cursor, tmp);
    csr_dedupe<<<blocks_of(nv + 1, 256), 256, 0, st>>>(nv, off, deg, tmp, uniq);
    if (exclusive_scan(uniq, d_row, nv + 1, sums, st) != cudaSuccess) return CUE_ERR_CUDA;
    csr_compact<<<blocks_of(nv + 1, 256), 256, 0, st>>>(nv, off, uniq, d_row, tmp, d_col, d_m);
    return cudaGetLastError() == cudaSuccess ? CUE_OK : CUE_ERR_CUDA;
}

size_t cue_bfs_workspace_bytes(int32_t nv)
{
    if (nv < 0) return 0;
    return bfs_layout(nv).total;
}

int cue_bfs(int32_t nv, const int32_t *d_row, const int32_t *d_col, int32_t source, int32_t *d_level, void *d_ws,
            size_t ws_bytes, void *stream)
{
    if (nv < 0 || !d_row || !d_level || (nv > 0 && !d_col)) return CUE_ERR_ARG;
    const BfsLayout L = bfs_layout(nv);
    if (!ws_ok(d_ws, ws_bytes, L.total)) return CUE_ERR_WORKSPACE;
    if (nv == 0) return CUE_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *W = static_cast<unsigned char *>(d_ws);
    int maxb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxb, bfs_kernel, 256, 0) != cudaSuccess || maxb <= 0)
        return CUE_ERR_CUDA;
    const int grid = std::max(1, std::min(blocks_of(nv, 256), maxb * sm_count_g()));
    if (cudaMemsetAsync(W, 0, 768, st) != cudaSuccess) return CUE_ERR_CUDA;   // status, barrier, flags
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, bfs_kernel, (int)nv, d_row, d_col, (int)source, d_level,
                                       reinterpret_cast<uint8_t *>(W + L.F), reinterpret_cast<uint8_t *>(W + L.U),
                                       reinterpret_cast<int *>(W + L.flag), reinterpret_cast<PBar *>(W + L.bar),
                                       (unsigned)grid, kPersistSpinLimit, reinterpret_cast<unsigned *>(W + L.status));
    return e == cudaSuccess ? CUE_OK : CUE_ERR_CUDA;
}

int cue_graph_status(void *d_ws, void *stream)
{
    if (!d_ws) return CUE_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return CUE_ERR_CUDA;
    unsigned word = 0;
    if (cudaMemcpy(&word, d_ws, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess) return CUE_ERR_CUDA;
    if (word && cudaMemset(d_ws, 0, sizeof(word)) != cudaSuccess) return CUE_ERR_CUDA;
    return (word & kStatusTimeout) ? CUE_ERR_TIMEOUT : CUE_OK;
}

}  // extern "C"
