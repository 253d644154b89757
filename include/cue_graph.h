/*
 * cue_graph.h -- the connectivity stage: uniform-grid binning of points,
 * growth-cone / neuron connections, the adjacency list, breadth-first levels.
 *
 * Binning follows the paper's particle grid (Sec. 3.5, "Diffusion of guidance
 * molecules"): each point's grid cell is its hash, the (cell, point) pairs are
 * sorted, and one thread per sorted entry marks where a cell's entries start
 * and end (the paper's identifyCellStart; Table 1).  The sort is this
 * library's own (count, scan, scatter, then each cell's ids in order), so the
 * output is deterministic.  Connections (Sec. 3.3): a growth cone and a neuron
 * connect when their squared distance is below the square of the radius sum;
 * each cone tests the neurons of the 3^dim cells around its own.  The
 * adjacency list is Fig. 4's vertex-head array V_a into one edge array E_a.
 * The traversal is Fig. 5's level-synchronous breadth-first search with one
 * thread per vertex, run as one cooperative launch whose levels are separated
 * by a bounded grid barrier.
 *
 * All arrays are caller-owned device memory; sizes and grid shapes are host
 * values.  Calls are asynchronous on `stream` (a cudaStream_t, NULL = the
 * default stream).  Errors: CUE_ERR_ARG, CUE_ERR_WORKSPACE, CUE_ERR_CUDA
 * (codes of cue.h); a barrier wait that ran out is reported by
 * cue_graph_status.
 */
#ifndef CUE_GRAPH_H
#define CUE_GRAPH_H

#include "cue.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Workspace bytes of cue_bin_points for n points on a grid of n_cells cells. */
size_t cue_bin_workspace_bytes(int32_t n, int64_t n_cells);

/* Bin points pos [dim][n] (SoA floats) on the grid grid[0] x grid[1] (x grid[2])
 * of cubic cells of side `cell` anchored at the origin (coordinates outside
 * the grid are clamped into it):
 *   cell_of[i]      linear cell of point i, x fastest            (n int32)
 *   sorted_id[j]    points ordered by (cell, id)                 (n int32)
 *   cell_start[c]   first sorted index of cell c, -1 if empty    (n_cells int32)
 *   cell_end[c]     one past its last, -1 if empty               (n_cells int32)
 * dim is 2 or 3 (grid[2] ignored in 2D).  Cells with many points are sorted
 * by one thread each (quadratic in the cell's count). */
int cue_bin_points(int32_t dim, int32_t n, const float *d_pos, float cell, const int32_t *grid,
                   int32_t *d_cell_of, int32_t *d_sorted_id, int32_t *d_cell_start, int32_t *d_cell_end,
                   void *d_ws, size_t ws_bytes, void *stream);

/* Connections of the active growth cones pos [dim][n_cones] (owner[a] = the
 * neuron cone a grows from) to the neurons npos [dim][n_neurons] binned by
 * cue_bin_points with the same cell and grid (cell >= radius, so the 3^dim
 * cells around a cone hold every neuron within reach): every pair with
 * |x - y|^2 < radius^2 other than a cone and its own neuron is written as
 * (src, dst) = (owner, neuron), in no particular order, at most `cap` of them;
 * *d_count receives the full count (set, not added).  d_active may be NULL. */
int cue_connect(int32_t dim, int32_t n_cones, const float *d_pos, const int32_t *d_owner,
                const uint8_t *d_active, int32_t n_neurons, const float *d_npos, float radius, float cell,
                const int32_t *grid, const int32_t *d_sorted_id, const int32_t *d_cell_start,
                const int32_t *d_cell_end, int32_t cap, int32_t *d_src, int32_t *d_dst, int32_t *d_count,
                void *stream);

/* Workspace bytes of cue_csr_build for nv vertices and up to ne_cap edges. */
size_t cue_csr_workspace_bytes(int32_t nv, int32_t ne_cap);

/* Adjacency list of the distinct edges among the first min(*d_ne, ne_cap) of
 * (src[k], dst[k]) (the count is read on the device, so the output of
 * cue_connect can be passed without a host round trip): row[v] .. row[v+1]
 * index col (nv + 1 and ne_cap int32), each row's targets ascending; *d_m
 * receives the number of distinct edges.  Vertices outside [0, nv) are
 * skipped. */
int cue_csr_build(int32_t nv, int32_t ne_cap, const int32_t *d_ne, const int32_t *d_src, const int32_t *d_dst,
                  int32_t *d_row, int32_t *d_col, int32_t *d_m, void *d_ws, size_t ws_bytes, void *stream);

/* Workspace bytes of cue_bfs for nv vertices. */
size_t cue_bfs_workspace_bytes(int32_t nv);

/* Breadth-first levels from `source` over the adjacency list (row, col):
 * level[v] = the number of edges on a shortest path, -1 when unreachable. */
int cue_bfs(int32_t nv, const int32_t *d_row, const int32_t *d_col, int32_t source, int32_t *d_level,
            void *d_ws, size_t ws_bytes, void *stream);

/* Synchronise `stream`; CUE_ERR_TIMEOUT if a barrier wait of the last cue_bfs
 * in this workspace ran out (each cue_bfs clears the flag when it starts;
 * this call clears it too), else CUE_OK. */
int cue_graph_status(void *d_ws, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CUE_GRAPH_H */
