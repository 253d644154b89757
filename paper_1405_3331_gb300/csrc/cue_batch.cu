// cue_batch.cu -- C ABI of batched runs (include/cue_batch.h): many
// independent 2D instances stepped by the persistent engine of k_persist.cu,
// by one launch per step, or by the temporally blocked kernel of k_blocked.cu,
// optionally through a captured CUDA graph, with a measuring autotuner for the
// run mode, the launch shape and the temporal depth.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <new>
#include <vector>

#include "cue_batch.h"
#include "cue_internal.h"

namespace cue {
namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace: [status | ctrl 256 | barrier 512 | per-instance cone counters |
// instance table | work list | source coordinates and binned sources | backup
// (optional)].
struct BatchLayout {
    size_t ctrl, bar, counters, inst, items, step_items, src_xyz, backup, total;
    size_t items_cap;
    std::vector<size_t> xyz_off, ent_off, key_off, bk_field, bk_cone;   // per instance
    // temporally blocked mode (sized for the deepest accepted depth, which has the most tiles)
    bool blk_ok = false;
    size_t blk_inst, blk_items, blk_chunks, blk_counts, blk_ids, blk_done;
    size_t blk_tiles_cap = 0, blk_chunks_cap = 0, blk_bins_cap = 0;
};

constexpr int kBlockedMaxDepth = 8;    // deepest temporal block of the batched blocked mode
constexpr int kBlockedDefaultDepth = 4;

size_t inst_cells(const cue_instance &I) { return (size_t)I.pitch * I.params.ny; }

// Every instance can run on the temporally blocked kernel: its depth-8 tile
// geometry exists, its sources fit the tile lists, and TMA maps can be made.
bool blocked_capable(int n, const cue_instance *in)
{
    if (!encode_field_map_available()) return false;
    for (int i = 0; i < n; ++i) {
        const cue_instance &I = in[i];
        if (I.params.dim != 2 || I.n_src > kBlockedMaxSrc || I.pitch % 4 != 0) return false;
        cue_params p = I.params;
        p.nz = 1;
        FieldDesc f;
        ConeDesc c;
        FusedGeom g;
        if (make_descs(p, I.cone, f, c) != CUE_OK) return false;
        if (!blocked_geometry(f, c.step_len, c.stop_r2, I.n_axons > 0, kBlockedMaxDepth, g)) return false;
        if ((long long)g.ntx * g.nty * std::max(I.n_axons, 1) > (1LL << 30)) return false;
    }
    return true;
}

BatchLayout batch_layout(int n, const cue_instance *in, bool backup)
{
    BatchLayout L;
    size_t off = 256;
    L.ctrl = off;
    off += 256;
    L.bar = off;
    off += 256;
    L.counters = off;                                    // one cone-update counter per instance
    off += align256(sizeof(unsigned long long) * (size_t)n);
    L.inst = off;
    off += align256(sizeof(PInst) * (size_t)n);
    L.items_cap = 0;
    for (int i = 0; i < n; ++i)
        L.items_cap += (size_t)persist_tiles(in[i].params.nx, in[i].params.ny, 1) +
                       (size_t)(std::max(in[i].n_axons, 0) + kPersistConeChunk - 1) / kPersistConeChunk;
    L.items = off;
    off += align256(sizeof(PItem) * std::max<size_t>(L.items_cap, 1));
    L.step_items = off;                                  // the same items, cone chunks first, for one launch per step
    off += align256(sizeof(PItem) * std::max<size_t>(L.items_cap, 1));
    L.src_xyz = off;
    L.xyz_off.resize(n);
    L.ent_off.resize(n);
    L.key_off.resize(n);
    for (int i = 0; i < n; ++i) {
        const size_t ns = (size_t)std::max(in[i].n_src, 0);
        L.xyz_off[i] = off;
        off += align256(sizeof(float) * 3 * ns);
        L.ent_off[i] = off;                              // sources binned to field tiles
        off += align256(sizeof(PSrc) * ns);
        L.key_off[i] = off;
        off += align256(sizeof(int) * ns);
    }
    // blocked mode: instance table, (instance, tile) items, cone chunks for the binning,
    // bin counts (two rounds) and bins that hold every cone of an instance (two rounds)
    L.blk_ok = blocked_capable(n, in);
    if (L.blk_ok) {
        for (int i = 0; i < n; ++i) {
            FieldDesc f;
            ConeDesc c;
            cue_params p = in[i].params;
            p.nz = 1;
            FusedGeom g;
            make_descs(p, in[i].cone, f, c);
            blocked_geometry(f, c.step_len, c.stop_r2, in[i].n_axons > 0, kBlockedMaxDepth, g);
            const size_t tiles = (size_t)g.ntx * g.nty;
            L.blk_tiles_cap += tiles;
            L.blk_bins_cap += tiles * (size_t)std::max(in[i].n_axons, 0);
            L.blk_chunks_cap += (size_t)(std::max(in[i].n_axons, 0) + 255) / 256;
        }
        L.blk_inst = off;
        off += align256(sizeof(BInst) * (size_t)n);
        L.blk_items = off;
        off += align256(sizeof(int2) * std::max<size_t>(L.blk_tiles_cap, 1));
        L.blk_chunks = off;
        off += align256(sizeof(int2) * std::max<size_t>(L.blk_chunks_cap, 1));
        L.blk_counts = off;
        off += align256(sizeof(int) * 2 * std::max<size_t>(L.blk_tiles_cap, 1));
        L.blk_ids = off;
        off += align256(sizeof(int) * 2 * std::max<size_t>(L.blk_bins_cap, 1));
        L.blk_done = off;
        off += 256;
    }
    L.backup = off;
    L.bk_field.resize(n);
    L.bk_cone.resize(n);
    if (backup) {
        for (int i = 0; i < n; ++i) {
            L.bk_field[i] = off;
            off += align256(sizeof(float) * inst_cells(in[i]));
            L.bk_cone[i] = off;                          // pos, dir ([2][n] each), active (n bytes)
            off += align256(sizeof(float) * 4 * (size_t)in[i].n_axons + (size_t)in[i].n_axons);
        }
    }
    L.total = off;
    return L;
}

bool instance_ok(const cue_instance &I)
{
    if (!params_ok(&I.params) || !cone_ok(&I.cone)) return false;
    if (I.params.dim != 2) return false;
    if (I.pitch < I.params.nx || I.pitch % 4 != 0) return false;
    if (!I.field_a || !I.field_b || I.field_a == I.field_b) return false;
    if (!aligned16(I.field_a) || !aligned16(I.field_b) || (I.src_map && !aligned16(I.src_map))) return false;
    if (I.n_src < 0 || I.n_axons < 0) return false;
    if (I.n_src > 0 && (!I.src_cell || !I.src_emit)) return false;
    if (I.n_axons > 0 && (!I.pos || !I.dir || !I.active)) return false;
    if ((long long)I.pitch * I.params.ny > (1LL << 31) - 1) return false;
    return true;
}

// Source node coordinates of one instance for the cones' stop test.
__global__ void batch_source_coords(int nx, int ny, float h, const int32_t *__restrict__ cell, int n_src, float *xyz,
                                    unsigned *status)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_src) return;
    const long long c = cell[s];
    if (c < 0 || c >= (long long)nx * ny) {
        flag_status(status, kStatusBounds);
        xyz[s] = xyz[n_src + s] = xyz[2 * n_src + s] = 3.0e38f;
        return;
    }
    xyz[s] = (float)(c % nx) * h;
    xyz[n_src + s] = (float)(c / nx) * h;
    xyz[2 * n_src + s] = 0.0f;
}

}  // namespace
}  // namespace cue

using namespace cue;

struct cue_batch {
    int n = 0;
    std::vector<cue_instance> in;
    std::vector<PInst> insts;
    BatchLayout L;
    bool has_backup = false;
    unsigned char *ws = nullptr;
    cudaStream_t stream = nullptr;
    int rows = 0, bpsm = 0;          // options (0 = library choice)
    int mode = 0;                    // option: 0 library choice (persistent unless tuned), 1 persistent, 2 per step,
                                     // 3 temporally blocked
    int depth = 0;                   // option: steps per blocked launch (0 = library choice)
    int blk_K = 0;                   // depth the blocked tables were staged for (0 = not staged)
    int blk_items = 0, blk_chunks = 0, blk_tiles = 0;
    size_t blk_bins = 0;
    int rows_used = 0;
    int n_items = 0;
    int n_step_tiles = 0, n_step_chunks = 0;
    bool list_ready = false;
    bool use_graph = false;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = -1;
    int graph_grid = 0;
    long long step = 0;
    int cur = 0;
    int grid = 0;

    unsigned *status() const { return reinterpret_cast<unsigned *>(ws); }
    unsigned long long *counters() const { return reinterpret_cast<unsigned long long *>(ws + L.counters); }
    PCtrl *ctrl() const { return reinterpret_cast<PCtrl *>(ws + L.ctrl); }
    PBar *bar() const { return reinterpret_cast<PBar *>(ws + L.bar); }
    PInst *d_inst() const { return reinterpret_cast<PInst *>(ws + L.inst); }
    PItem *d_items() const { return reinterpret_cast<PItem *>(ws + L.items); }
    PItem *d_step_items() const { return reinterpret_cast<PItem *>(ws + L.step_items); }
    bool per_step() const { return mode == 2; }
    bool blocked() const { return mode == 3; }
    int blocked_depth() const { return depth > 0 ? depth : kBlockedDefaultDepth; }
    BInst *d_binst() const { return reinterpret_cast<BInst *>(ws + L.blk_inst); }
    int2 *d_blk_items() const { return reinterpret_cast<int2 *>(ws + L.blk_items); }
    int2 *d_blk_chunks() const { return reinterpret_cast<int2 *>(ws + L.blk_chunks); }
    int *blk_counts() const { return reinterpret_cast<int *>(ws + L.blk_counts); }
    int *blk_ids() const { return reinterpret_cast<int *>(ws + L.blk_ids); }
    int *blk_done() const { return reinterpret_cast<int *>(ws + L.blk_done); }
};

namespace {

int sm_count_b()
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

void drop_graph(cue_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_steps = -1;
}

int pick_rows_b(const cue_batch *b)
{
    if (b->rows > 0) return b->rows;
    long long tiles4 = 0;
    for (int i = 0; i < b->n; ++i) tiles4 += persist_tiles(b->in[i].params.nx, b->in[i].params.ny, 4);
    const long long target = 2LL * sm_count_b();
    int rows = 4;
    while (rows > 1 && tiles4 * (4 / rows) < target) rows /= 2;
    return rows;
}

// (Re)build the instance table and the work list for the current rows (the
// persistent kernel's tiles have at most 4 rows per warp; the per-step
// launches stream 8 or 16 as well).
int stage_list(cue_batch *b)
{
    const int rows = b->per_step() ? pick_rows_b(b) : std::min(pick_rows_b(b), 4);
    if (b->list_ready && rows == b->rows_used) return CUE_OK;
    for (int i = 0; i < b->n; ++i) persist_fill(b->insts[i], b->insts[i].f, rows, b->in[i].pitch);
    std::vector<PItem> items;
    persist_items(b->insts, items);
    if (items.size() > b->L.items_cap) return CUE_ERR_WORKSPACE;
    // one launch per step: every cone chunk, then every tile (instance by instance)
    std::vector<PItem> step_items;
    step_items.reserve(items.size());
    for (const PItem &w : items)
        if (w.idx < 0) step_items.push_back(w);
    const int n_chunks = (int)step_items.size();
    for (const PItem &w : items)
        if (w.idx >= 0) step_items.push_back(w);
    if (cudaMemcpyAsync(b->d_inst(), b->insts.data(), sizeof(PInst) * b->insts.size(), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess ||
        (!items.empty() && cudaMemcpyAsync(b->d_items(), items.data(), sizeof(PItem) * items.size(),
                                           cudaMemcpyHostToDevice, b->stream) != cudaSuccess) ||
        (!step_items.empty() && cudaMemcpyAsync(b->d_step_items(), step_items.data(),
                                                sizeof(PItem) * step_items.size(), cudaMemcpyHostToDevice,
                                                b->stream) != cudaSuccess) ||
        persist_bin_sources(b->d_inst(), b->n, b->d_items(), (int)items.size(), b->status(), b->stream) !=
            cudaSuccess ||
        persist_bin_sources(b->d_inst(), b->n, b->d_step_items(), (int)step_items.size(), b->status(),
                            b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)       // the host vectors are released below
        return CUE_ERR_CUDA;
    b->n_items = (int)items.size();
    b->n_step_chunks = n_chunks;
    b->n_step_tiles = (int)step_items.size() - n_chunks;
    b->rows_used = rows;
    b->list_ready = true;
    drop_graph(b);
    return CUE_OK;
}

// The blocked mode's instance table (tensor maps of both buffers, tile geometry
// for depth K, first tile and first bin of each instance), its (instance, tile)
// items instance by instance, and the cone chunks of the binning launch.
int stage_blocked(cue_batch *b, int K)
{
    if (!b->L.blk_ok) return CUE_ERR_ARG;
    if (b->blk_K == K) return CUE_OK;
    std::vector<BInst> bi(b->n);
    std::vector<int2> items, chunks;
    std::vector<int> order_key;
    int tile_base = 0;
    size_t bin_base = 0;
    for (int i = 0; i < b->n; ++i) {
        const cue_instance &I = b->in[i];
        const PInst &P = b->insts[i];
        BInst &B = bi[i];
        std::memset(static_cast<void *>(&B), 0, sizeof(BInst));
        FusedGeom g;
        if (!blocked_geometry(P.f, P.c.step_len, P.c.stop_r2, I.n_axons > 0, K, g)) return CUE_ERR_ARG;
        if (!encode_field_map(&B.map[0], I.field_a, I.params.nx, I.params.ny, I.pitch) ||
            !encode_field_map(&B.map[1], I.field_b, I.params.nx, I.params.ny, I.pitch))
            return CUE_ERR_CUDA;
        B.f = P.f;
        B.c = P.c;
        B.g = g;
        B.field[0] = I.field_a;
        B.field[1] = I.field_b;
        B.rate_map = I.src_map;
        B.src_cell = I.src_cell;
        B.src_emit = I.src_emit;
        B.src_xyz = P.src_xyz;
        B.pos = I.pos;
        B.dir = I.dir;
        B.active = I.active;
        B.counter = P.counter;
        B.pitch = I.pitch;
        B.n_src = I.n_src;
        B.n_axons = I.n_axons;
        B.tile_base = tile_base;
        B.bin_base = bin_base;
        const int tiles = g.ntx * g.nty;
        for (int t = 0; t < tiles; ++t) {
            items.push_back(make_int2(i, t));
            // the order key: the sweep instantiation the tile runs (rate map, y wall, right
            // wall inside a float4 group), so that the CTAs resident together run the same
            // code (measured on the 512-instance workload: 547 -> 682 G node updates/s, the
            // instruction fetch of eight unrolled sweeps being the first stall); then the
            // tile's expected cone load (the instance's cones over its tiles, in powers of
            // two), heaviest first so that no crowded tile is left for a group's last wave
            // (-> 704).  Tiles whose cones take more than one round through global memory
            // per sub-step (over 768) run longest: they go first, ahead of every group, so
            // that none of them is left for the launch's tail (-> 752)
            const int tx = t % g.ntx, ty = t / g.ntx;
            const int ox = blocked_x(g, I.params.nx).origin(tx), oy = blocked_y(g, I.params.ny).origin(ty);
            const int nx = I.params.nx, ny = I.params.ny;
            const bool ragged = (nx & 3) != 0 && ox + kBlockedTileW > nx - 1;
            const bool wall = oy <= -1 || oy + kBlockedTileRows - 1 >= ny;
            const int load = std::max(I.n_axons, 0) / tiles;
            int lclass = 0;
            while ((1 << lclass) <= load && lclass < 30) ++lclass;
            const int cls = (I.src_map ? 4 : 0) | (wall ? 2 : 0) | (ragged ? 1 : 0);
            order_key.push_back(load > kFusedBinCap + kBlockedThreads ? 30 - lclass : ((cls + 1) << 8) | (30 - lclass));
        }
        for (int a0 = 0; a0 < I.n_axons; a0 += 256) chunks.push_back(make_int2(i, a0));
        tile_base += tiles;
        bin_base += (size_t)tiles * (size_t)std::max(I.n_axons, 0);
    }
    if (items.size() > b->L.blk_tiles_cap || chunks.size() > b->L.blk_chunks_cap || bin_base > b->L.blk_bins_cap)
        return CUE_ERR_WORKSPACE;
    {   // items in key order, instance order kept within a key (the tiles are independent
        // within a launch, so the order changes no result)
        std::vector<size_t> idx(items.size());
        for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
        std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return order_key[x] < order_key[y]; });
        std::vector<int2> sorted(items.size());
        for (size_t k = 0; k < idx.size(); ++k) sorted[k] = items[idx[k]];
        items.swap(sorted);
    }
    if (cudaMemcpyAsync(b->d_binst(), bi.data(), sizeof(BInst) * bi.size(), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        (!items.empty() && cudaMemcpyAsync(b->d_blk_items(), items.data(), sizeof(int2) * items.size(),
                                           cudaMemcpyHostToDevice, b->stream) != cudaSuccess) ||
        (!chunks.empty() && cudaMemcpyAsync(b->d_blk_chunks(), chunks.data(), sizeof(int2) * chunks.size(),
                                            cudaMemcpyHostToDevice, b->stream) != cudaSuccess) ||
        cudaMemsetAsync(b->blk_done(), 0, sizeof(int), b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)       // the host vectors are released below
        return CUE_ERR_CUDA;
    b->blk_items = (int)items.size();
    b->blk_chunks = (int)chunks.size();
    b->blk_tiles = tile_base;
    b->blk_bins = bin_base;
    b->blk_K = K;
    drop_graph(b);
    return CUE_OK;
}

// A run of the blocked mode: both rounds of bin counts cleared, the bin round
// reset, every cone binned, then ceil(nsteps / K) blocked launches (the last
// one shorter); the kernels advance the step control themselves.
cudaError_t launch_blocked(cue_batch *b, int nsteps)
{
    const int K = b->blk_K;
    cudaError_t e = cudaMemsetAsync(b->blk_counts(), 0, sizeof(int) * 2 * (size_t)std::max(b->blk_tiles, 1),
                                    b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&b->ctrl()->pad[0], 0, sizeof(uint32_t), b->stream);
    if (e == cudaSuccess)
        e = blocked_bin(b->d_binst(), b->d_blk_chunks(), b->blk_chunks, b->blk_counts(), b->blk_ids(), b->blk_bins,
                        b->blk_tiles, b->ctrl(), b->stream);
    for (int done = 0; e == cudaSuccess && done < nsteps; done += K)
        e = blocked_launch(b->d_binst(), b->d_blk_items(), b->blk_items, std::min(K, nsteps - done), b->ctrl(),
                           b->blk_counts(), b->blk_ids(), b->blk_bins, b->blk_tiles, b->blk_done(), b->status(),
                           b->stream);
    b->grid = b->blk_items;
    return e;
}

cudaError_t launch_direct(cue_batch *b, int nsteps)
{
    if (b->blocked()) return launch_blocked(b, nsteps);
    if (b->per_step()) {
        b->grid = b->n_step_tiles;
        return step_launch(b->d_inst(), b->d_step_items(), b->n_step_chunks, b->d_step_items() + b->n_step_chunks,
                           b->n_step_tiles, b->n_items == b->n_step_chunks + b->n_step_tiles ? b->d_items() : nullptr,
                           b->rows_used, nsteps, b->ctrl(), b->stream);
    }
    return persist_launch(b->d_inst(), b->d_items(), b->n_items, nsteps, 0, 0, b->bar(), b->bpsm, 0, 0, b->status(),
                          b->stream, &b->grid, b->ctrl());
}

int run_graph(cue_batch *b, int nsteps)
{
    if (!b->graph || b->graph_steps != nsteps) {
        drop_graph(b);
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CUE_ERR_CUDA;
        cudaError_t e = launch_direct(b, nsteps);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return CUE_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return CUE_ERR_CUDA;
        }
        b->graph_steps = nsteps;
        b->graph_grid = b->grid;
    }
    b->grid = b->graph_grid;
    return cudaGraphLaunch(b->graph, b->stream) == cudaSuccess ? CUE_OK : CUE_ERR_CUDA;
}

// Longest graph of the per-step mode (one node per time step): longer runs
// replay it, then launch the remainder directly.  The buffer parity and the
// step counter live on the device, so the pieces chain without new arguments.
constexpr int kStepGraphMax = 1024;

int run_batch(cue_batch *b, int nsteps)
{
    int rc = b->blocked() ? stage_blocked(b, b->blocked_depth()) : stage_list(b);
    if (rc != CUE_OK) return rc;
    if (b->use_graph && (b->per_step() || b->blocked()) && nsteps > kStepGraphMax) {
        for (int i = 0; i < nsteps / kStepGraphMax && rc == CUE_OK; ++i) rc = run_graph(b, kStepGraphMax);
        if (rc == CUE_OK && nsteps % kStepGraphMax)
            rc = launch_direct(b, nsteps % kStepGraphMax) == cudaSuccess ? CUE_OK : CUE_ERR_CUDA;
    } else if (b->use_graph) {
        rc = run_graph(b, nsteps);
    } else {
        rc = launch_direct(b, nsteps) == cudaSuccess ? CUE_OK : CUE_ERR_CUDA;
    }
    if (rc != CUE_OK) return rc;
    b->step += nsteps;
    if (b->blocked()) {             // one buffer flip per blocked launch, K steps each, per run piece
        const int K = b->blk_K;
        long long flips = 0;
        if (b->use_graph && nsteps > kStepGraphMax)
            flips = (long long)(nsteps / kStepGraphMax) * ((kStepGraphMax + K - 1) / K) +
                    (nsteps % kStepGraphMax + K - 1) / K;
        else
            flips = (nsteps + K - 1) / K;
        b->cur ^= (int)(flips & 1);
    } else {
        b->cur ^= (nsteps & 1);
    }
    return CUE_OK;
}

// Save / restore every instance's current state (field, pos, dir, active),
// the step control block and the cone counter.
int save_state(cue_batch *b, std::vector<unsigned long long> &counter)
{
    counter.assign(b->n, 0ull);
    for (int i = 0; i < b->n; ++i) {
        const cue_instance &I = b->in[i];
        const float *f = b->cur ? I.field_b : I.field_a;
        unsigned char *bf = b->ws + b->L.bk_field[i], *bc = b->ws + b->L.bk_cone[i];
        const size_t na = (size_t)I.n_axons;
        if (cudaMemcpyAsync(bf, f, sizeof(float) * inst_cells(I), cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
            return CUE_ERR_CUDA;
        if (na && (cudaMemcpyAsync(bc, I.pos, sizeof(float) * 2 * na, cudaMemcpyDeviceToDevice, b->stream) !=
                       cudaSuccess ||
                   cudaMemcpyAsync(bc + sizeof(float) * 2 * na, I.dir, sizeof(float) * 2 * na,
                                   cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
                   cudaMemcpyAsync(bc + sizeof(float) * 4 * na, I.active, na, cudaMemcpyDeviceToDevice, b->stream) !=
                       cudaSuccess))
            return CUE_ERR_CUDA;
    }
    if (cudaMemcpyAsync(counter.data(), b->counters(), sizeof(unsigned long long) * b->n, cudaMemcpyDeviceToHost,
                        b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return CUE_ERR_CUDA;
    return CUE_OK;
}

int restore_state(cue_batch *b, int cur, long long step, const std::vector<unsigned long long> &counter)
{
    for (int i = 0; i < b->n; ++i) {
        const cue_instance &I = b->in[i];
        float *f = cur ? I.field_b : I.field_a;
        const unsigned char *bf = b->ws + b->L.bk_field[i], *bc = b->ws + b->L.bk_cone[i];
        const size_t na = (size_t)I.n_axons;
        if (cudaMemcpyAsync(f, bf, sizeof(float) * inst_cells(I), cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
            return CUE_ERR_CUDA;
        if (na && (cudaMemcpyAsync(I.pos, bc, sizeof(float) * 2 * na, cudaMemcpyDeviceToDevice, b->stream) !=
                       cudaSuccess ||
                   cudaMemcpyAsync(I.dir, bc + sizeof(float) * 2 * na, sizeof(float) * 2 * na,
                                   cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
                   cudaMemcpyAsync(I.active, bc + sizeof(float) * 4 * na, na, cudaMemcpyDeviceToDevice, b->stream) !=
                       cudaSuccess))
            return CUE_ERR_CUDA;
    }
    PCtrl c{};
    c.cur = cur;
    c.step0 = (uint32_t)step;
    if (cudaMemcpyAsync(b->ctrl(), &c, sizeof(c), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->counters(), counter.data(), sizeof(unsigned long long) * b->n, cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return CUE_ERR_CUDA;
    b->cur = cur;
    b->step = step;
    return CUE_OK;
}

}  // namespace

extern "C" {

size_t cue_batch_workspace_bytes(int32_t n, const cue_instance *inst, int32_t with_backup)
{
    if (n <= 0 || !inst) return 0;
    for (int i = 0; i < n; ++i)
        if (inst[i].params.dim != 2 || inst[i].pitch < inst[i].params.nx || inst[i].n_src < 0 ||
            inst[i].n_axons < 0)
            return 0;
    return batch_layout(n, inst, with_backup != 0).total;
}

cue_batch *cue_batch_create(int32_t n, const cue_instance *inst, void *d_ws, size_t ws_bytes, void *stream,
                            int32_t *err)
{
    int32_t dummy;
    if (!err) err = &dummy;
    *err = CUE_ERR_ARG;
    if (n <= 0 || !inst) return nullptr;
    for (int i = 0; i < n; ++i)
        if (!instance_ok(inst[i])) return nullptr;
    std::vector<FieldDesc> fd(n);
    std::vector<ConeDesc> cd(n);
    for (int i = 0; i < n; ++i) {
        cue_params p = inst[i].params;
        p.nz = 1;
        if (make_descs(p, inst[i].cone, fd[i], cd[i]) != CUE_OK) {
            *err = CUE_ERR_UNSTABLE;
            return nullptr;
        }
    }
    const BatchLayout with = batch_layout(n, inst, true), without = batch_layout(n, inst, false);
    const bool backup = ws_bytes >= with.total;
    if (!d_ws || ws_bytes < without.total || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) {
        *err = CUE_ERR_WORKSPACE;
        return nullptr;
    }
    cue_batch *b = new (std::nothrow) cue_batch();
    if (!b) return nullptr;
    b->n = n;
    b->in.assign(inst, inst + n);
    b->L = backup ? with : without;
    b->has_backup = backup;
    b->ws = static_cast<unsigned char *>(d_ws);
    b->stream = static_cast<cudaStream_t>(stream);
    b->insts.resize(n);
    for (int i = 0; i < n; ++i) {
        const cue_instance &I = inst[i];
        PInst &P = b->insts[i];
        P = PInst{};
        P.f = fd[i];
        P.c = cd[i];
        P.field0 = I.field_a;
        P.field1 = I.field_b;
        P.map = I.src_map;
        P.src_cell = I.src_cell;
        P.src_emit = I.src_emit;
        P.src_xyz = reinterpret_cast<const float *>(b->ws + b->L.xyz_off[i]);
        P.n_src = I.n_src;
        P.n_axons = I.n_axons;
        P.pos = I.pos;
        P.dir = I.dir;
        P.active = I.active;
        P.status = b->status();
        P.counter = b->counters() + i;
        P.src_ent = I.n_src > 0 ? reinterpret_cast<PSrc *>(b->ws + b->L.ent_off[i]) : nullptr;
        P.src_key = I.n_src > 0 ? reinterpret_cast<int *>(b->ws + b->L.key_off[i]) : nullptr;
    }
    cudaError_t e = cudaMemsetAsync(b->ws, 0, b->L.inst, b->stream);     // status, ctrl, barrier, counters
    for (int i = 0; e == cudaSuccess && i < n; ++i) {
        const cue_instance &I = inst[i];
        if (I.n_src > 0 && cd[i].stop_r2 >= 0.0f) {
            batch_source_coords<<<(I.n_src + 127) / 128, 128, 0, b->stream>>>(
                I.params.nx, I.params.ny, I.params.h, I.src_cell, I.n_src,
                reinterpret_cast<float *>(b->ws + b->L.xyz_off[i]), b->status());
            e = cudaGetLastError();
        }
    }
    int rc = e == cudaSuccess ? stage_list(b) : CUE_ERR_CUDA;
    if (rc != CUE_OK) {
        *err = rc;
        delete b;
        return nullptr;
    }
    *err = CUE_OK;
    return b;
}

int cue_batch_run(cue_batch *b, int32_t nsteps)
{
    if (!b || nsteps < 0) return CUE_ERR_ARG;
    if (b->step + nsteps > 0xFFFFFFFFLL) return CUE_ERR_STATE;
    for (int done = 0; done < nsteps;) {
        const int k = std::min(nsteps - done, kPersistMaxSteps);
        const int rc = run_batch(b, k);
        if (rc != CUE_OK) return rc;
        done += k;
    }
    return CUE_OK;
}

int cue_batch_autotune(cue_batch *b, int32_t probe_steps, int32_t *rows_out, int32_t *bpsm_out, double *ms_out)
{
    if (!b || probe_steps <= 0) return CUE_ERR_ARG;
    if (!b->has_backup) return CUE_ERR_WORKSPACE;
    std::vector<unsigned long long> counter;
    const int cur0 = b->cur;
    const long long step0 = b->step;
    int rc = save_state(b, counter);
    if (rc != CUE_OK) return rc;
    const int keep_rows = b->rows, keep_bpsm = b->bpsm, keep_mode = b->mode, keep_depth = b->depth;
    const bool keep_graph = b->use_graph;
    b->use_graph = false;
    const int maxb = std::max(1, std::min(3, persist_max_blocks_per_sm()));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CUE_ERR_CUDA;
    double best = 1e30;
    int best_rows = 0, best_b = 0, best_mode = 1, best_depth = 0;
    auto probe = [&](int mode, int rows, int bb, int depth) {
        b->rows = rows;
        b->bpsm = bb;
        b->mode = mode;
        b->depth = depth;
        rc = run_batch(b, std::min(probe_steps, 2 * std::max(depth, 1)));   // warm: stages the tables, first touch
        if (rc == CUE_OK) rc = restore_state(b, cur0, step0, counter);
        if (rc != CUE_OK) return;
        float ms = 0.f;
        if (cudaEventRecord(e0, b->stream) != cudaSuccess) rc = CUE_ERR_CUDA;
        if (rc == CUE_OK) rc = run_batch(b, probe_steps);
        if (rc == CUE_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = CUE_ERR_CUDA;
        if (rc == CUE_OK && ms / probe_steps < best) {
            best = ms / probe_steps;
            best_rows = rows;
            best_b = bb;
            best_mode = mode;
            best_depth = depth;
        }
        if (rc == CUE_OK) rc = restore_state(b, cur0, step0, counter);
    };
    const int rows_c[5] = {1, 2, 4, 8, 16};
    // candidates: the persistent launch (rows 1, 2, 4 x blocks per SM 1..maxb), one
    // launch per step (rows 2..16; "blocks per SM" 0), and the temporally blocked
    // launch (depth 2, 4, 8; rows and blocks 0) where every instance can take it
    for (int ri = 0; ri < 5 && rc == CUE_OK; ++ri)
        for (int bb = 0; bb <= maxb && rc == CUE_OK; ++bb) {
            if ((bb == 0 && rows_c[ri] == 1) || (bb > 0 && rows_c[ri] > 4)) continue;
            probe(bb == 0 ? 2 : 1, rows_c[ri], bb, 0);
        }
    for (int K = 2; b->L.blk_ok && K <= kBlockedMaxDepth && rc == CUE_OK; K *= 2) probe(3, 0, 0, K);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->use_graph = keep_graph;
    if (rc != CUE_OK) {
        b->rows = keep_rows;
        b->bpsm = keep_bpsm;
        b->mode = keep_mode;
        b->depth = keep_depth;
        return rc;
    }
    b->rows = best_rows;
    b->bpsm = best_b;
    b->mode = best_mode;
    b->depth = best_depth;
    b->list_ready = false;
    drop_graph(b);
    if (rows_out) *rows_out = best_rows;
    if (bpsm_out) *bpsm_out = best_b;
    if (ms_out) *ms_out = best;
    rc = stage_list(b);
    if (rc == CUE_OK && b->blocked()) rc = stage_blocked(b, b->blocked_depth());
    return rc;
}

int cue_batch_set_state(cue_batch *b, int64_t step, int32_t cur)
{
    if (!b || (cur != 0 && cur != 1) || step < 0 || step > 0xFFFFFFFFLL) return CUE_ERR_ARG;
    PCtrl c{};
    c.cur = cur;
    c.step0 = (uint32_t)step;
    if (cudaMemcpyAsync(b->ctrl(), &c, sizeof(c), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return CUE_ERR_CUDA;
    b->cur = cur;
    b->step = step;
    return CUE_OK;
}

int cue_batch_set_option(cue_batch *b, int32_t option, int64_t value)
{
    if (!b) return CUE_ERR_ARG;
    switch (option) {
    case CUE_BOPT_ROWS:
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16) return CUE_ERR_ARG;
        b->rows = (int)value;
        b->list_ready = b->list_ready && pick_rows_b(b) == b->rows_used;
        drop_graph(b);
        return CUE_OK;
    case CUE_BOPT_BLOCKS:
        if (value < 0 || value > 8) return CUE_ERR_ARG;
        b->bpsm = (int)value;
        drop_graph(b);
        return CUE_OK;
    case CUE_BOPT_GRAPH:
        if (value != 0 && value != 1) return CUE_ERR_ARG;
        b->use_graph = value != 0;
        if (!b->use_graph) drop_graph(b);
        return CUE_OK;
    case CUE_BOPT_MODE:
        if (value < 0 || value > 3) return CUE_ERR_ARG;
        if (value == 3 && !b->L.blk_ok) return CUE_ERR_ARG;
        b->mode = (int)value;
        drop_graph(b);
        return CUE_OK;
    case CUE_BOPT_DEPTH:
        if (value < 0 || value > kBlockedMaxDepth) return CUE_ERR_ARG;
        b->depth = (int)value;
        drop_graph(b);
        return CUE_OK;
    default:
        return CUE_ERR_ARG;
    }
}

int cue_batch_get_option(const cue_batch *b, int32_t option, int64_t *value)
{
    if (!b || !value) return CUE_ERR_ARG;
    switch (option) {
    case CUE_BOPT_ROWS: *value = b->rows_used; return CUE_OK;
    case CUE_BOPT_BLOCKS: *value = b->bpsm; return CUE_OK;
    case CUE_BOPT_GRAPH: *value = b->use_graph ? 1 : 0; return CUE_OK;
    case CUE_BINFO_ITEMS: *value = b->n_items; return CUE_OK;
    case CUE_BINFO_STEP: *value = b->step; return CUE_OK;
    case CUE_BINFO_CUR: *value = b->cur; return CUE_OK;
    case CUE_BINFO_GRID: *value = b->grid; return CUE_OK;
    case CUE_BOPT_MODE: *value = b->blocked() ? 3 : b->per_step() ? 2 : 1; return CUE_OK;
    case CUE_BOPT_DEPTH: *value = b->blocked_depth(); return CUE_OK;
    case CUE_BINFO_BLOCKED: *value = b->L.blk_ok ? 1 : 0; return CUE_OK;
    default: return CUE_ERR_ARG;
    }
}

int cue_batch_status(cue_batch *b)
{
    if (!b) return CUE_ERR_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return CUE_ERR_CUDA;
    unsigned word = 0;
    if (cudaMemcpy(&word, b->status(), sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess) return CUE_ERR_CUDA;
    if (word && cudaMemset(b->status(), 0, sizeof(unsigned)) != cudaSuccess) return CUE_ERR_CUDA;
    if (word & kStatusNonFinite) return CUE_ERR_NONFINITE;
    if (word & kStatusTimeout) return CUE_ERR_TIMEOUT;
    if (word & kStatusBounds) return CUE_ERR_BOUNDS;
    return cuda_err(cudaGetLastError());
}

int cue_batch_cone_updates(cue_batch *b, uint64_t *count)
{
    if (!b || !count) return CUE_ERR_ARG;
    std::vector<unsigned long long> v(b->n, 0ull);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return CUE_ERR_CUDA;
    if (cudaMemcpy(v.data(), b->counters(), sizeof(unsigned long long) * b->n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return CUE_ERR_CUDA;
    if (cudaMemset(b->counters(), 0, sizeof(unsigned long long) * b->n) != cudaSuccess) return CUE_ERR_CUDA;
    unsigned long long tot = 0;
    for (unsigned long long x : v) tot += x;
    *count = tot;
    return CUE_OK;
}

void cue_batch_destroy(cue_batch *b)
{
    if (!b) return;
    drop_graph(b);
    delete b;
}

}  // extern "C"
