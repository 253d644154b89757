/*
 * cue_batch.h -- many independent 2D cue-field / growth-cone simulations of
 * uneven sizes and parameters stepped together.
 *
 * Each instance is the model of cue.h (Sec. 5.2 field update with no-flux
 * walls, decay and point sources; Sec. 3.5 growth-cone steering with Philox
 * noise; Sec. 3.3-3.4 stop tests), with its own grid, physics, sources and
 * cones.  The paper steps one environment; running many in one launch is this
 * library's own addition.  All instances' field tiles and cone chunks form
 * one work list, instance by instance.  A cue_batch_run call runs it in one
 * of three modes (CUE_BOPT_MODE; the autotuner picks): one cooperative launch
 * in which every block takes items each step and the blocks meet at a
 * bounded grid barrier between steps; one ordinary launch per step with one
 * item per block; or temporally blocked launches, each advancing every
 * instance's field tiles and their cones several steps in shared memory.  Any
 * of them can be replayed from a captured CUDA graph.
 * Per node and per cone the arithmetic is cue.h's plain path, so an instance
 * here evolves bit for bit as it would alone (source cells distinct).
 *
 * Layout: instance i's field buffers hold ny rows of `pitch[i]` floats
 * (pitch >= nx, a multiple of 4, 16-byte aligned buffers); columns
 * nx..pitch-1 are padding the library never changes.  Source cells are
 * linear node indices x + nx*y (as in cue.h), cone state is SoA [2][n].
 *
 * Ownership: every device buffer, the workspace and the stream belong to the
 * caller and must outlive the batch.  Calls are asynchronous on the stream;
 * two calls on one batch must not overlap.
 *
 * Errors: negative CUE_ERR_* codes of cue.h; device-side conditions (non-
 * finite values, out-of-range source cells, a barrier wait that ran out) are
 * latched on the device and reported by cue_batch_status.
 */
#ifndef CUE_BATCH_H
#define CUE_BATCH_H

#include "cue.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cue_batch cue_batch;   /* opaque, host-side */

/* One instance: host struct of device pointers and sizes. */
typedef struct {
    cue_params params;        /* dim must be 2; boundary 0                          */
    cone_params cone;
    int32_t pitch;            /* row pitch of both field buffers, floats           */
    float *field_a;           /* C^n on entry (buffer 0), ny * pitch floats         */
    float *field_b;           /* second buffer, same size                           */
    const int32_t *src_cell;  /* n_src node indices x + nx*y                        */
    const float *src_emit;    /* n_src emissions per step                           */
    int32_t n_src;
    const float *src_map;     /* nullable: rate map, ny * pitch floats (adds dt*M)  */
    float *pos, *dir;         /* [2][n_axons] each                                  */
    uint8_t *active;          /* n_axons                                            */
    int32_t n_axons;
} cue_instance;

/* Device workspace bytes for a batch of n instances (256-byte aligned).
 * with_backup != 0 adds room for one copy of every instance's state, which
 * cue_batch_autotune needs (it measures candidates and restores the state). */
size_t cue_batch_workspace_bytes(int32_t n, const cue_instance *inst, int32_t with_backup);

/* Create a batch.  inst[0..n) is copied (the device buffers are not).  Stages
 * the instance table and the work list in the workspace on `stream` (a
 * cudaStream_t, NULL = default stream).  Returns NULL and sets *err on error:
 * CUE_ERR_ARG (bad instance, dim != 2, pitch, alignment), CUE_ERR_UNSTABLE
 * (1 - 4 alpha - lambda dt < 0 for an instance), CUE_ERR_WORKSPACE,
 * CUE_ERR_CUDA. */
cue_batch *cue_batch_create(int32_t n, const cue_instance *inst, void *d_ws, size_t ws_bytes, void *stream,
                            int32_t *err);

/* Advance every instance by nsteps coupled steps (cones on C^n, then
 * C^n -> C^{n+1}).  One cooperative launch (CUE_BOPT_MODE 1), one or two
 * launches per step (mode 2), or (mode 3) the cones binned to field tiles and
 * then one temporally blocked launch per CUE_BOPT_DEPTH steps -- each field
 * tile of each instance loaded once into shared memory with its halo (tiles
 * aligned to the instance's walls, no halo beyond a wall) and advanced that
 * many steps there with its cones -- or one graph replay of
 * those when CUE_BOPT_GRAPH is on (the graph is captured at the first call
 * with a given nsteps and replayed afterwards; the step counter, buffer
 * parity and bin round live on the device, so a replay needs no new
 * arguments). */
int cue_batch_run(cue_batch *b, int32_t nsteps);

/* Time each candidate launch shape (rows per thread 1, 2, 4 x blocks per SM
 * 1..3 of the persistent launch, rows 2, 4, 8, 16 of one launch per step, and
 * temporal depths 2, 4, 8 of the blocked mode when CUE_BINFO_BLOCKED is 1) on
 * probe_steps steps from the current state, restoring the state after every
 * candidate, and keep the fastest (CUE_BOPT_MODE and CUE_BOPT_DEPTH then say
 * which).  Needs the backup area (see cue_batch_workspace_bytes).
 * Synchronises the stream.  Writes the chosen rows and blocks per SM (both 0
 * for the blocked mode; blocks 0 alone: one launch per step) and the best
 * time per step (ms) when non-null. */
int cue_batch_autotune(cue_batch *b, int32_t probe_steps, int32_t *rows, int32_t *blocks_per_sm,
                       double *ms_per_step);

/* Set every instance's step counter and current buffer (0 = field_a), e.g. after
 * the caller has written new states into the buffers.  Asynchronous on the
 * stream.  CUE_ERR_ARG for cur not 0/1 or step outside [0, 2^32). */
int cue_batch_set_state(cue_batch *b, int64_t step, int32_t cur);

#define CUE_BOPT_ROWS    1    /* rows per thread of a field tile (1, 2, 4; 8 and 16 */
                              /* with one launch per step: the tile is streamed)    */
#define CUE_BOPT_BLOCKS  2    /* blocks per SM (1..8, capped by occupancy)          */
#define CUE_BOPT_GRAPH   3    /* 1: run through a captured CUDA graph; 0: direct    */
#define CUE_BOPT_MODE    4    /* 1: one persistent launch per run (grid barrier     */
                              /* between steps); 2: per step one launch over every  */
                              /* instance's cone chunks and one over every tile;    */
                              /* 3: temporally blocked, one launch per DEPTH steps  */
                              /* (CUE_ERR_ARG when CUE_BINFO_BLOCKED is 0);         */
                              /* 0: library choice (1 unless the autotuner picked)  */
#define CUE_BOPT_DEPTH   5    /* steps per launch of mode 3 (1..8; 0: library       */
                              /* choice, 4)                                         */
#define CUE_BINFO_ITEMS  16   /* work-list length (field tiles + cone chunks)       */
#define CUE_BINFO_STEP   17   /* steps taken so far (host mirror)                   */
#define CUE_BINFO_CUR    18   /* current buffer of every instance: 0 = field_a      */
                              /* (modes 1, 2 flip it every step, mode 3 once per    */
                              /* launch of DEPTH steps)                              */
#define CUE_BINFO_GRID   19   /* blocks of the last launch                          */
#define CUE_BINFO_BLOCKED 20  /* 1 when every instance can run in mode 3 (its depth-8 */
                              /* tile geometry exists and it has <= 256 sources)    */

int cue_batch_set_option(cue_batch *b, int32_t option, int64_t value);
int cue_batch_get_option(const cue_batch *b, int32_t option, int64_t *value);

/* Synchronise the stream; return and clear the latched device status. */
int cue_batch_status(cue_batch *b);

/* Number of active-cone updates since the last call (synchronises). */
int cue_batch_cone_updates(cue_batch *b, uint64_t *count);

/* Release the handle (not the caller's buffers); destroys a captured graph. */
void cue_batch_destroy(cue_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* CUE_BATCH_H */
