// cue_internal.h -- host-side definitions shared by the translation units of
// libcue.so (handle layout, workspace layout, kernel launchers).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>
#include <vector>

#include "cue.h"
#include "cue_device.cuh"

namespace cue {

// Workspace layout (all offsets 256-byte aligned):
//   [0,   256)  status word (unsigned) at 0, cone-update counter (u64) at 8
//   [256, ...)  source coordinates, FP32 [3][n_src]
//   [...]       fused-path scratch (two rounds each): per-tile cone counts,
//               per-tile bins of cone ids (bin_cap each), a spill list of
//               (cone, tile) for overfull tiles and its count.  n_tiles is an
//               upper bound over every tile geometry.  bin_cap is n_axons (a
//               tile's bin holds any number of its cones, so the spill list
//               stays empty) while the bins fit in kFusedBinBudget, else
//               kFusedBinCap.
constexpr int kFusedBinCap = 512;   // ids per tile bin when the bins cannot hold every cone (large grids)
constexpr size_t kFusedBinBudget = size_t(256) << 20;   // bytes of bins (both rounds) that buy bin_cap = n_axons

struct WorkspaceLayout {
    size_t status_off = 0;
    size_t src_xyz_off = 0;
    size_t bin_count_off = 0;    // 2 x n_tiles int32 (double-buffered counts)
    size_t bin_ctl_off = 0;      // spill counts (2 int32) and a finished-tile counter
    size_t bin_list_off = 0;     // 2 x n_tiles x bin_cap int32 (cone ids by tile)
    size_t spill_off = 0;        // 2 x n_axons int2 (cone, tile) that did not fit their bin
    size_t persist_off = 0;      // persistent path: barrier, two instance records, work list
    size_t persist_items_cap = 0;
    size_t persist_src_off = 0;  // persistent path: binned sources (PSrc) and their tile keys
    size_t inter_off = 0;        // blocked 3D path: scratch copy of the field's intermediate step (0: none)
    size_t total = 0;
    int n_tiles = 0;
    int bin_cap = 0;             // cone ids per tile bin
};

// Tile geometry of the fused path.
struct FusedGeom {
    int W, R;            // loaded columns, rows
    int HX, HY;          // halo columns (multiple of 4), rows
    int TX, TY;          // interior columns, rows
    int ntx, nty;        // tiles per axis
    int K;               // temporal depth
    int ctas_per_sm;
    int local_stop;      // 1: the halo covers the source-stop radius, test tile sources only
};

// Box geometry of the temporally blocked 3D path (k_fused3d.cu): column tiles
// of 128 x TY nodes in x-y, chunks of ZC planes in z, one CTA per box.
struct Fused3Geom {
    int TY = 0;
    int ntx = 0, nty = 0;
    int nchunk = 0, ZC = 0;
    int boxes = 0;
};
// The geometry depends on the grid only (the workspace's bins are sized by it).
bool fused3d_geometry(const cue_params &p, Fused3Geom &g);

WorkspaceLayout workspace_layout(const cue_params &p, int n_src, int n_axons);
// Device descriptors of one simulation (CUE_ERR_UNSTABLE when the explicit step is unstable).
int make_descs(const cue_params &params, const cone_params &cone, FieldDesc &f, ConeDesc &c);
bool params_ok(const cue_params *p);
bool cone_ok(const cone_params *c);
bool aligned16(const void *p);
int cuda_err(cudaError_t e);

// ---- persistent path (k_persist.cu) ----
constexpr int kPersistThreads = 256;          // 32 lanes x 8 warps
constexpr int kPersistWarps = 8;
constexpr int kPersistConeChunk = 256;        // cones per work item (one per thread)
constexpr long long kPersistSpinLimit = 1LL << 24;   // polls (~32 ns apart) before a barrier gives up
constexpr int kPersistMaxSteps = 1 << 20;            // steps per launch (longer runs take several)

// A point source binned to its field tile: node offset y * pitch + x (-1 when
// the cell is outside the grid) and the source's index.
struct PSrc {
    int off;
    int k;
};
// One instance of the persistent engine (device-side table entry).
struct PInst {
    FieldDesc f;
    ConeDesc c;
    float *field0, *field1;
    const float *map;                 // dense rate map or null
    const int32_t *src_cell;
    const float *src_emit;
    const float *src_xyz;
    int n_src;
    int n_axons;
    float *pos, *dir;
    uint8_t *active;
    unsigned *status;
    unsigned long long *counter;
    float *traj_field;                // trajectory mode: [nsteps + 1][cells] (else null)
    float *traj_cone;                 // trajectory mode: [nsteps + 1][pos, dir][2][n] (else null)
    PSrc *src_ent;                    // n_src binned sources, sorted by (tile, index), or null
    int *src_key;                     // their tiles (same order)
    size_t cells;                     // pitch * ny: elements of one field buffer
    int ntx, rows;                    // field tiles per tile row, rows per thread
    int pitch;                        // row pitch in floats (multiple of 4, >= nx)
};
struct PItem {
    int inst;
    int idx;                          // >= 0: field tile; < 0: cone chunk ~idx
    int src_begin, src_n;             // field tile: its range of the instance's binned sources
                                      // (src_n < 0: sources not binned, the tile scans them)
};
constexpr int kPersistBinCap = 4096;  // instances with more sources scan them per tile
struct PBar {
    unsigned long long count;   // arrivals since the launch began (only grows)
    int abort;
    unsigned pad;
};
// Step counter and buffer parity kept on the device (batched runs), so that a
// captured launch can be replayed without new arguments.
struct PCtrl {
    int cur;
    uint32_t step0;
    uint32_t pad[2];
};

struct Sim {
    cue_params params;
    cone_params cone;
    FieldDesc fd;
    ConeDesc cd;
    float *field[2];
    const int32_t *src_cell;
    const float *src_emit;
    int n_src;
    const float *src_map;
    float *pos, *dir;
    uint8_t *active;
    int n_axons;
    unsigned char *ws;
    size_t ws_bytes;
    WorkspaceLayout wl;
    cudaStream_t stream;
    int64_t field_step = 0, cone_step = 0;
    int cur = 0;
    int path = CUE_PATH_AUTO;
    int temporal_depth = 0;
    int rows_per_thread = 0;     // plain 2D field kernel; 0 = heuristic
    uint64_t launches = 0;
    bool vec4 = false;           // nx % 4 == 0 and 16-byte aligned buffers
    bool src_xyz_ready = false;

    // dominant-kernel timing (CUE_OPT_TIME_KERNEL): a ring of event pairs
    bool time_kernel = false;
    int time_period = 1;          // time every time_period-th launch
    long long time_seen = 0;      // dominant-kernel launches seen while timing
    bool timing_now = false;      // the current launch is bracketed
    std::vector<cudaEvent_t> ev_start, ev_stop;
    size_t ev_next = 0, ev_live = 0;
    double timed_ms = 0.0;
    uint64_t timed_launches = 0;

    // resident and cluster paths
    bool resident_used = false;
    bool cluster_used = false;
    int cluster_opt = 0;          // option: CTAs per cluster (0 = library picks, 8 or 16)
    mutable int cluster_pick = -1;  // cached cluster_ctas() for cluster_opt (-1 = not yet asked)
    int cluster_last = 0;         // CTAs of the last cluster launch

    // adjoint trace (cue_adjoint_trace): copies of the forward states the backward pass reads
    float *adj_trace_field = nullptr;   // [max_states][cells]
    float *adj_trace_cone = nullptr;    // [max_states][pos, dir][dim * n_axons]
    int64_t adj_trace_cap = 0;

    // persistent path
    bool persist_ready = false, persist_used = false;
    int persist_rows = 0;         // option (0 = heuristic)
    int persist_rows_used = 0;
    int persist_bpsm = 0;         // option: blocks per SM (0 = default)
    int persist_phantom = 0;      // diagnostic option: barrier arrivals that never come
    long long persist_limit = 0;  // option: polls before a bounded wait gives up (0 = default)
    int persist_n_items = 0;
    int persist_grid = 0;

    // fused path
    // helper CTAs for crowded tiles: the total need the last run reported, read back
    // without blocking (pinned word + event) and applied to the next run
    bool adapt_helpers = true;    // off for handles that must not allocate (sim_run_static)
    int *help_host = nullptr;     // pinned host words: the run's largest need, the two round slots
    cudaEvent_t help_ev = nullptr;
    bool help_pending = false;
    int help_next = 0;            // helpers the next run launches
    int help_last = 0;            // helpers of the last fused launch (CUE_INFO_HELPERS)
    FusedGeom geom{};
    bool geom_ready = false;
    // point sources per fused tile region: the source cells on the host (copied once,
    // when there are more than a tile's list holds) and the verdict for one depth
    mutable std::vector<int32_t> src_cells_host;
    mutable int src_fit_K = -1;
    mutable bool src_fit_ok = false;
    bool fused_used = false;
    long long bin_round = 0;
    alignas(64) unsigned char tmap[2][128];   // CUtensorMap per field buffer (as TMA source)
    alignas(64) unsigned char tmap3[2][128];  // 3D plane maps of the field buffers
    bool tmap3_ready = false;
    // temporally blocked 3D path
    Fused3Geom geom3{};
    bool geom3_ready = false;
    alignas(64) unsigned char tmap3b[2][128]; // 3D plane maps with the blocked path's box

    int *bin_count() const { return reinterpret_cast<int *>(ws + wl.bin_count_off); }
    int *bin_ctl() const { return reinterpret_cast<int *>(ws + wl.bin_ctl_off); }
    int *bin_list() const { return reinterpret_cast<int *>(ws + wl.bin_list_off); }
    int2 *spill() const { return reinterpret_cast<int2 *>(ws + wl.spill_off); }
    unsigned *status() const { return reinterpret_cast<unsigned *>(ws + wl.status_off); }
    unsigned long long *cone_counter() const
    {
        return reinterpret_cast<unsigned long long *>(ws + wl.status_off + 8);
    }
    float *src_xyz() const { return reinterpret_cast<float *>(ws + wl.src_xyz_off); }
    float *inter3() const { return wl.inter_off ? reinterpret_cast<float *>(ws + wl.inter_off) : nullptr; }
    PBar *persist_bar() const { return reinterpret_cast<PBar *>(ws + wl.persist_off); }
    PInst *persist_inst() const { return reinterpret_cast<PInst *>(ws + wl.persist_off + 256); }
    PItem *persist_items() const
    {
        return reinterpret_cast<PItem *>(ws + wl.persist_off + 256 + ((2 * sizeof(PInst) + 255) & ~(size_t)255));
    }
    PSrc *persist_src_ent() const { return reinterpret_cast<PSrc *>(ws + wl.persist_src_off); }
    int *persist_src_key() const
    {
        return reinterpret_cast<int *>(ws + wl.persist_src_off + ((sizeof(PSrc) * (size_t)n_src + 255) & ~(size_t)255));
    }
};

bool persist_supported(const Sim &s);
int persist_max_blocks_per_sm();
int persist_tiles(int nx, int ny, int rows);
void persist_fill(PInst &I, const FieldDesc &f, int rows, int pitch);
void persist_items(const std::vector<PInst> &insts, std::vector<PItem> &items);
// ctrl null: cur0 / step0 are used; else they are read from *ctrl at the start,
// and *ctrl is advanced by nsteps after the launch (a second, one-thread kernel).
// Bin every instance's sources to its field tiles and give each field-tile item
// its range (after the table and the list are in device memory).
cudaError_t persist_bin_sources(PInst *d_insts, int n_inst, PItem *d_items, int n_items, unsigned *status,
                                cudaStream_t stream);
cudaError_t persist_launch(const PInst *d_insts, const PItem *d_items, int n_items, int nsteps, int cur0,
                           uint32_t step0, PBar *d_bar, int blocks_per_sm, int phantom, long long limit,
                           unsigned *status, cudaStream_t stream, int *grid_out, PCtrl *ctrl = nullptr);
// A batch's steps as ordinary launches (no grid barrier): per step one launch
// over the cone-chunk items d_chunks, then one over the field-tile items
// d_tiles (tiles of `rows` rows per warp, as the instance table says); for
// rows > 4 (streamed tiles) instead one launch over d_mixed, the same
// n_chunks + n_tiles items in instance order.  Buffers and the Philox step
// from *ctrl plus the step index, and *ctrl advanced by nsteps at the end.
// The non-finite check runs on the last step.
cudaError_t step_launch(const PInst *d_insts, const PItem *d_chunks, int n_chunks, const PItem *d_tiles,
                        int n_tiles, const PItem *d_mixed, int rows, int nsteps, PCtrl *ctrl, cudaStream_t stream);
// Runs nsteps on the persistent path when selected (or AUTO) and supported:
// CUE_OK / negative error when it ran, 1 when the caller should fall back.
int run_persist_if_supported(Sim &s, int nsteps);
// Coupled steps storing every state (trajectory slot 0 holds the start).
int run_persist_trajectory(Sim &s, float *traj_field, float *traj_cone, uint32_t step0, int nsteps);

// ---- shared-memory resident path for small 2D grids (k_resident.cu) ----
constexpr int kResThreads = 1024;         // one block: field warps first, then one warp per 32 cones
constexpr int kResMaxCones = 256;         // at most 8 cone warps (24 warps stay on the field)
constexpr int kResMaxSources = 1024;
bool resident_supported(const Sim &s);
// Runs nsteps on the resident path when selected (or AUTO) and supported:
// CUE_OK / negative error when it ran, 1 when the caller should fall back.
int run_resident_if_supported(Sim &s, int nsteps);

// ---- small 2D grids spread over a thread-block cluster (k_cluster.cu) ----
constexpr int kClusterSize = 8;           // CTAs per cluster at the portable size, one band of rows each
constexpr int kClusterSizeLarge = 16;     // the non-portable size, where the device can schedule it
constexpr int kClusterThreads = 1024;     // threads per CTA: field warps first, then one warp per 32 cones
constexpr int kClusterMaxConeWarps = 16;  // cones per CTA at most 512 (16 warps stay on the field)
constexpr int kClusterMaxSources = 1024;
bool cluster_supported(const Sim &s);
// CTAs per cluster the cluster path launches for this simulation (its option,
// else the larger size that fits and the device can schedule); 0 = unsupported.
int cluster_ctas(const Sim &s);
// Whether AUTO takes the cluster path: supported, at least 4,096 nodes, at most
// 128 cones and 16,384 nodes per CTA (the shapes on which it measured faster
// than the single-block and persistent kernels).
bool cluster_preferred(const Sim &s);
// Runs nsteps on the cluster path when selected (or AUTO) and supported:
// CUE_OK / negative error when it ran, 1 when the caller should fall back.
int run_cluster_if_supported(Sim &s, int nsteps);

// ---- fused, temporally blocked path (k_fused.cu) ----
constexpr int kMaxTemporalDepth = 16;
int fused_tile_count(const cue_params &p);   // tiles of the fused path (0 if unsupported)
bool fused_supported(const Sim &s);
// Runs nsteps on the fused path when selected and supported: returns CUE_OK or
// a negative error when it ran, 1 when the caller should use the plain path.
int run_fused_if_supported(Sim &s, int nsteps);
// Same for field-only steps (cue_step).
int field_fused_if_supported(Sim &s, int nsteps);

// ---- temporally blocked 3D path (k_fused3d.cu): two steps per launch ----
bool fused3d_supported(const Sim &s);
// Runs nsteps (coupled when `cones`, else field only) on the blocked 3D path
// when selected (or AUTO) and supported: CUE_OK / negative error when it ran,
// 1 when the caller should use the one-launch-per-step kernels.
int run_fused3d_if_supported(Sim &s, int nsteps, bool cones);

// Bracket a launch of the dominant kernel with timing events (no-ops when off).
void timing_begin(Sim &s);
void timing_end(Sim &s);

// ---- temporally blocked batch mode (k_blocked.cu) ----
constexpr int kBlockedMaxSrc = 256;   // point sources per instance on this mode
constexpr int kBlockedTileW = 256;    // loaded columns and rows of a blocked-mode tile
constexpr int kBlockedTileRows = 96;
constexpr int kBlockedThreads = 256;   // threads of a blocked-mode CTA
// One instance of a batch in the blocked mode (device table; the tensor maps
// give the struct their 128-byte alignment, which the workspace's 256-byte
// offsets keep).
struct BInst {
    CUtensorMap map[2];               // TMA source maps of field_a / field_b (nx x ny, row pitch)
    FieldDesc f;
    ConeDesc c;
    FusedGeom g;                      // tile geometry for the launch's depth
    float *field[2];
    const float *rate_map;            // [ny][pitch] or null
    const int32_t *src_cell;
    const float *src_emit;
    const float *src_xyz;
    float *pos, *dir;
    uint8_t *active;
    unsigned long long *counter;
    size_t bin_base;                  // this instance's first bin (tile 0) in one round of ids
    int pitch, n_src, n_axons, tile_base;
};
// Tile geometry of the temporally blocked kernels for depth K (false if none).
bool fused_geometry(const FieldDesc &f, float step_len, float stop_r2, bool cones, int K, FusedGeom &g);

// Wall-aligned tiling of one axis of n nodes for the batch's blocked mode.  A
// tile that holds a wall needs no halo on that side (the wall node is its own
// missing neighbour), so the first tile starts at the wall and the last ends at
// it: load extent W, halo H, interior T = W - 2H between two tiles, and `ghost`
// rows kept beyond a wall (1 in y, where the sweep reads a ghost row; 0 in x,
// where the lanes' wall flags stand in).  First interior F = W - ghost - H.
// n <= W - 2 ghost: one tile from -ghost.  Otherwise tile 0 holds [0, F), tile
// k >= 1 starts at F + (k - 1) T with origin start - H, and the last tile holds
// the rest (at most F nodes, so its loaded region reaches its wall and ghost).
struct AxisTiles {
    int n, W, H, ghost;
    __host__ __device__ int first() const { return W - ghost - H; }
    __host__ __device__ int inner() const { return W - 2 * H; }
    __host__ __device__ bool single() const { return n <= W - 2 * ghost; }
    __host__ __device__ int count() const
    {
        if (single()) return 1;
        const int rest = n - 2 * first();
        return 2 + (rest > 0 ? (rest + inner() - 1) / inner() : 0);
    }
    __host__ __device__ int start(int k) const { return k == 0 ? 0 : first() + (k - 1) * inner(); }
    __host__ __device__ int origin(int k) const { return k == 0 ? -ghost : start(k) - H; }
    __host__ __device__ int end(int k) const { return k + 1 >= count() ? n : start(k + 1); }
    __host__ __device__ int index(int i) const      // tile of node i (0 <= i < n)
    {
        if (single() || i < first()) return 0;
        const int k = 1 + (i - first()) / inner();
        const int last = count() - 1;
        return k < last ? k : last;
    }
};
__host__ __device__ inline AxisTiles blocked_x(const FusedGeom &g, int nx) { return AxisTiles{nx, g.W, g.HX, 0}; }
__host__ __device__ inline AxisTiles blocked_y(const FusedGeom &g, int ny) { return AxisTiles{ny, g.R, g.HY, 1}; }
// The fused geometry with the batch's wall-aligned tile counts in ntx / nty.
bool blocked_geometry(const FieldDesc &f, float step_len, float stop_r2, bool cones, int K, FusedGeom &g);
// Encode a 2D TMA source map of an nx x ny FP32 field with rows `pitch` floats apart.
bool encode_field_map(void *map128, float *base, int nx, int ny, int pitch);
bool encode_field_map_available();
size_t blocked_smem_bytes();
cudaError_t blocked_bin(const BInst *d_insts, const int2 *d_chunks, int n_chunks, int *counts, int *ids,
                        size_t bin_total, int total_tiles, const PCtrl *ctrl, cudaStream_t stream);
cudaError_t blocked_launch(const BInst *d_insts, const int2 *d_items, int n_items, int K, PCtrl *ctrl, int *counts,
                           int *ids, size_t bin_total, int total_tiles, int *done, unsigned *status,
                           cudaStream_t stream);

// A handle that allocates nothing, not even the pinned word of the helper readback.
void sim_no_host_alloc(cue_sim *h);
// ---- coupled steps without the public entry point's checks (cue_api.cu)
int run_coupled(Sim &s, int nsteps);
// ---- adjoint (k_adjoint.cu)
size_t adjoint_workspace_bytes(const cue_params &p, int n_src, int n_axons, int nsteps, int ckpt_every);
int run_adjoint(Sim &s, const float *targets, int nsteps, int ckpt_every, void *ws, size_t ws_bytes, float *gD,
                float *gl, float *gsrc, float *gmap, float *loss);
// The endpoint loss of the handle's current cone state (one launch).
cudaError_t launch_endpoint_loss(Sim &s, const float *targets, float *loss);

// ---- launchers (each returns cudaGetLastError() after its launches) ----
// One field step Cin -> Cout.  With `sources_done` non-null the kernel may also
// add the point sources; *sources_done tells whether it did.
cudaError_t launch_field_step(Sim &s, const float *Cin, float *Cout, bool *sources_done = nullptr);
// Field step followed by the point sources (in the same kernel where it can).
cudaError_t launch_field_and_sources(Sim &s, const float *Cin, float *Cout);
cudaError_t launch_sources(Sim &s, float *Cout);
cudaError_t launch_src_xyz(Sim &s);
cudaError_t launch_cone_step(Sim &s, const float *C, uint32_t step);
cudaError_t launch_cone_step_io(Sim &s, const float *C, uint32_t step, const float *pin, const float *din,
                                float *pout, float *dout);
// 3D field step through the TMA plane pipeline (k_field3d.cu)
bool field3d_tma_prepare(Sim &s);
// cones_done (optional): the field blocks also step the cones on the input
// buffer (cone step index s.cone_step) when one thread each covers them, and
// *cones_done says whether they did; sources_done (optional): the field
// blocks add the point sources when there are at most kTma3BlockSources of
// them, and *sources_done says whether they did.
constexpr int kTma3BlockSources = 1024;
cudaError_t launch_field3d_tma(Sim &s, int in_buffer, float *Cout, bool *cones_done = nullptr,
                               bool *sources_done = nullptr);

}  // namespace cue
