/*
 * cue.h -- C ABI of libcue.so: GB300 (sm_103a) cue-field diffusion and
 * growth-cone steering.
 *
 * The model follows Mihut, Morgan & Kaiser, "GPU Simulation of Axon Growth
 * and Guidance through Cue Diffusion": guidance cues live on a fixed
 * Eulerian grid (Sec. 5.2) and are emitted by sources placed pseudo-randomly
 * with their own diffusion rates (Sec. 4.3); each axon's growth cone advances
 * a fixed distance per step along a direction that is steered by vector
 * addition of its current direction and the cue direction it senses
 * (Sec. 3.5, Eq. 6-7), with Gaussian noise from a stateless per-thread
 * counter-based generator (Sec. 5.1, Sec. 3.2 Box-Muller); cones stop when
 * they leave the simulation bounds (Sec. 3.4) or come within a radius of a
 * source, tested on squared distances (Sec. 3.3).
 *
 * One time step n -> n+1:
 *   cones (read C^n):  g   = multilinear interpolation at p of the node
 *                            central-difference gradients of C^n
 *                      v   = w_prev d + w_grad g/|g| + w_noise xi
 *                      d'  = v/|v|;  p' = p + step_len d'
 *                      stop if p' leaves [0,(N-1)h]^dim (or clamp), or if
 *                      |p' - x_k|^2 <= stop_radius^2 for a source node x_k
 *   field:             C^{n+1}_i = C^n_i + alpha sum_{axis nbrs j}(C_j - C_i)
 *                                  - lambda dt C^n_i  (+ e_k at source k)
 *                                  (+ dt M_i for a dense rate map M)
 *                      alpha = D dt / h^2, missing neighbours at the walls
 *                      contribute nothing (no-flux).
 *   noise:             Philox-4x32-10, key = (seed lo, seed hi),
 *                      counter = (axon, step, 0, 0), Box-Muller on the words.
 *
 * Conventions for every call below.
 *   - Layout: fields are dense FP32 arrays, x fastest:
 *     index = i + nx (j + ny k), node (i,j,k) at (i h, j h, k h).
 *     Cone state is structure-of-arrays: pos[c*n_axons + a] is coordinate c
 *     of cone a (same for dir); active[a] is 0 or 1.
 *   - Ownership: every buffer is allocated and owned by the caller (for
 *     example with PyTorch) and must stay valid until cue_destroy.  The
 *     library allocates no device memory: all its scratch lives in the
 *     caller's workspace (cue_workspace_bytes).  The handle is host memory
 *     owned by the library and freed by cue_destroy.
 *   - Streams: every call is asynchronous on the stream given to cue_init
 *     (or cue_set_stream); only cue_status synchronises.
 *   - Errors: calls return CUE_OK (0) or a negative CUE_ERR_* code and never
 *     throw.  Device-side problems (non-finite values, out-of-range source
 *     cells, a bounded wait that ran out) are recorded in a status word in
 *     the workspace and reported by cue_status.
 */
#ifndef CUE_H
#define CUE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define CUE_OK               0
#define CUE_ERR_ARG         -1  /* invalid argument (null pointer, bad size, bad enum)      */
#define CUE_ERR_UNSTABLE    -2  /* D dt / h^2 > 1/(2 dim) or lambda dt outside [0, 1]     */
#define CUE_ERR_CUDA        -3  /* a CUDA runtime call failed                               */
#define CUE_ERR_NONFINITE   -4  /* a kernel produced a NaN or Inf                           */
#define CUE_ERR_TIMEOUT     -5  /* a bounded device-side wait gave up                       */
#define CUE_ERR_BOUNDS      -6  /* a source cell index outside the grid was skipped         */
#define CUE_ERR_WORKSPACE   -7  /* workspace missing, too small or misaligned               */
#define CUE_ERR_STATE       -8  /* call order violated (e.g. sim_run with cone/field steps
                                   out of step)                                             */
#define CUE_ERR_SCRATCH     -9  /* the problem needs more scratch than sim_run_static's
                                   fixed device array holds                                 */

/* ---- parameters -------------------------------------------------------- */
typedef struct {
    int32_t dim;            /* 2 or 3                                                  */
    int32_t nx, ny, nz;     /* nodes per axis, each >= 2 (nz ignored when dim == 2)    */
    float h;                /* node spacing, > 0                                       */
    float D;                /* diffusion coefficient, >= 0                             */
    float lambda;           /* decay rate, >= 0                                        */
    float dt;               /* time step, > 0                                          */
    int32_t boundary;       /* 0 = no-flux walls (the only value accepted)             */
} cue_params;

typedef struct {
    float w_prev;           /* weight of the previous direction                        */
    float w_grad;           /* weight of the normalised sensed gradient                */
    float w_noise;          /* weight of the Gaussian noise vector                     */
    float step_len;         /* distance advanced per step (same units as h)           */
    float stop_radius;      /* stop within this distance of a source node; <= 0: off   */
    float grad_eps;         /* |g| <= grad_eps counts as no gradient (default 1e-15)   */
    int32_t wall_mode;      /* 0 = stop when leaving the domain, 1 = clamp to it       */
    int32_t reserved;       /* must be 0                                               */
    uint64_t seed;          /* Philox key (low word, high word)                        */
} cone_params;

typedef struct cue_sim cue_sim;   /* opaque, host-side */

/* ---- options (cue_set_option) ------------------------------------------ */
#define CUE_OPT_PATH            1  /* value: CUE_PATH_*                                    */
#define CUE_OPT_TEMPORAL_DEPTH  2  /* value: steps fused per launch on the fused path (1..16),
                                      0 = library choice; on 3D handles 2 selects the
                                      blocked path under AUTO, other values the one-step
                                      kernel                                                */
#define CUE_OPT_ROWS_PER_THREAD 3  /* value: rows streamed per thread by the plain 2D field
                                      kernel (1..64), 0 = library choice                    */
#define CUE_OPT_TIME_KERNEL     4  /* value v >= 1: bracket every v-th launch of the dominant
                                      field kernel with CUDA events on the handle's stream,
                                      read back by cue_kernel_time; 0: off (default)        */
#define CUE_OPT_PERSIST_ROWS    5  /* value: rows per thread of a persistent-path field tile
                                      (1, 2 or 4), 0 = library choice                        */
#define CUE_OPT_PERSIST_BLOCKS  6  /* value: blocks per SM of the persistent launch (1..8,
                                      capped by occupancy), 0 = library choice (2)           */
#define CUE_OPT_WAIT_LIMIT      7  /* value: polls (about 32 ns apart) before a bounded
                                      device-side wait of the persistent path gives up and
                                      raises CUE_ERR_TIMEOUT; 0 = default (2^24)            */
#define CUE_OPT_BARRIER_PHANTOM 8  /* diagnostic: the persistent grid barrier also waits for
                                      this many arrivals that never come, so its bounded
                                      wait runs out (tests the timeout path); 0 = off       */
#define CUE_OPT_CLUSTER_CTAS    9  /* value: blocks per cluster of the cluster path: 0 = the
                                      library picks (16 where it fits and the device can
                                      schedule it, else 8), or 8 or 16; results do not
                                      depend on it                                           */
/* read-only values for cue_get_option */
#define CUE_INFO_LAST_PATH     16  /* CUE_PATH_*: path the last sim_run took                  */
#define CUE_INFO_TILE          17  /* fused tile interior: TX | TY << 16 (0 if not prepared);
                                      3D: the blocked path's column tile                     */
#define CUE_INFO_DEPTH         18  /* temporal depth the fused path runs with                 */
#define CUE_INFO_GRID          19  /* blocks of the last persistent or cluster launch         */
#define CUE_INFO_HELPERS       20  /* helper blocks of the last fused 2D launch: blocks that
                                      share out the cones of crowded tiles (sized from the
                                      crowding the previous run reported; 0 on the first)  */
#define CUE_PATH_AUTO   0          /* library picks: fused for 2D grids of at least one tile
                                      per SM; else cluster for 2D grids of at least 4096
                                      nodes with at most 128 cones and 16384 nodes per block;
                                      else resident; else persistent; else plain (3D: one
                                      launch per step)                                     */
#define CUE_PATH_PLAIN  1          /* one launch per half-step: cone kernel, field kernel
                                      (3D with nx % 4 == 0: one launch per step)           */
#define CUE_PATH_FUSED  2          /* temporally blocked field + cones in one kernel (2D:
                                      nx % 4 == 0, no rate map, at most 65536 sources and
                                      256 in any tile's loaded region); on 3D
                                      handles (nx % 4 == 0, step_len <= h, at most 512
                                      sources) two steps per launch, a run's odd last step
                                      on the one-step kernel                               */
#define CUE_PATH_PERSIST 3         /* 2D, nx % 4 == 0: one cooperative launch for the whole
                                      run; per step one pass over field tiles and cone
                                      chunks, then a bounded grid barrier                   */
#define CUE_PATH_RESIDENT 4        /* 2D, nx % 4 == 0, both field buffers within one block's
                                      shared memory (128^2: 128 KB), at most 256 cones and
                                      1024 sources: one block holds the grid in shared
                                      memory and the cones in registers for the whole call  */
#define CUE_PATH_CLUSTER 5         /* 2D, nx % 4 == 0, ny >= 2G, a band of ceil(ny / G) rows
                                      (both buffers plus two halo rows) within one block's
                                      shared memory, at most 512 G cones and 1024 sources: a
                                      cluster of G = 16 blocks (where the device schedules
                                      one; else G = 8, see CUE_OPT_CLUSTER_CTAS) holds the
                                      grid in distributed shared memory, one band each, for
                                      the whole call; one cluster barrier per step           */

/* Parameters of the SNR turn rule (Sec. 3.5, Eq. 5; 2D).  Inside the
 * detectable window c_min <= C(p) <= c_max the cone turns by `turn` radians to
 * the right (clockwise) when a draw from N(SNR, 1) is positive, else to the
 * left, with SNR = gain * mu * sqrt(gamma / (1 + gamma)^3) * sin(theta -
 * theta_NGF), gamma = C(p) / kd, mu = width * |grad C(p)| / C(p); outside the
 * window it keeps its direction.  C(p) is the bilinear cue value, grad C(p)
 * the sampled gradient of the vector-addition rule, the draw SNR plus the
 * cone's first Philox/Box-Muller normal of (cone, step). */
typedef struct {
    float gain;         /* Eq. 5's gain                                     */
    float width;        /* growth-cone width w                              */
    float kd;           /* concentration scale (> 0)                        */
    float c_min, c_max; /* detectable concentration window                  */
    float turn;         /* turn angle per step; the paper: pi/30            */
} cue_snr_params;

/* Bytes of device workspace the simulation needs (256-byte aligned). */
size_t cue_workspace_bytes(const cue_params *params, int32_t n_src, int32_t n_axons);

/*
 * Create a simulation handle over caller-owned device buffers.
 *   d_field_a   : C^n on entry (current buffer 0), nx*ny(*nz) floats
 *   d_field_b   : second field buffer of the same size (contents ignored)
 *   d_src_cell  : n_src int32 node indices (duplicates allowed; out-of-range
 *                 indices are skipped and reported as CUE_ERR_BOUNDS)
 *   d_src_emit  : n_src floats, emission added to the node every step
 *   d_src_map   : nullable; nx*ny(*nz) floats, rate map M (adds dt*M_i)
 *   d_pos,d_dir : dim*n_axons floats each (SoA), d_active: n_axons bytes
 *   d_workspace : >= cue_workspace_bytes(...) bytes, 256-byte aligned
 *   stream      : cudaStream_t (NULL = legacy default stream)
 * Returns CUE_OK, CUE_ERR_ARG, CUE_ERR_UNSTABLE, CUE_ERR_WORKSPACE or
 * CUE_ERR_CUDA.  On error *out is set to NULL.  Field and cone step
 * counters start at 0.
 */
int cue_init(cue_sim **out, const cue_params *params, const cone_params *cone,
             float *d_field_a, float *d_field_b,
             const int32_t *d_src_cell, const float *d_src_emit, int32_t n_src,
             const float *d_src_map,
             float *d_pos, float *d_dir, uint8_t *d_active, int32_t n_axons,
             void *d_workspace, size_t ws_bytes, void *stream);

/* Advance the field only, nsteps >= 0 times: the cue field on the fixed
 * Eulerian grid of Sec. 5.2, diffusing at its own rate from sources placed
 * pseudo-randomly (Sec. 4.3), written as the explicit update in the file
 * header (axis-neighbour stencil, decay, then the point emissions and the
 * rate map).  Increments the field step counter and flips the current buffer
 * once per step.  Errors: CUE_ERR_ARG (nsteps < 0), CUE_ERR_STATE (step
 * counter past 2^32 - 1), CUE_ERR_CUDA; device-side problems via
 * cue_status. */
int cue_step(cue_sim *sim, int32_t nsteps);

/* Advance the cones only, nsteps times, on the current field (held fixed):
 * the growth-cone steering of Sec. 3.5 -- the sensed cue gradient (Sec. 3.5,
 * the cone senses the concentration change across its width) is added to the
 * current direction (Eq. 6-7) together with Gaussian noise (Sec. 3.5, the
 * N(SNR,1) decision; Sec. 5.1 stateless counter-based generator; Sec. 3.2
 * Box-Muller), normalised, and the cone advances a fixed distance; it stops
 * when it leaves the bounds (Sec. 3.4) or comes within stop_radius of a
 * source, a squared-distance test (Sec. 3.3).  Step k uses Philox counter
 * step = cone counter + k.  Increments the cone step counter.  cone_step(1)
 * followed by cue_step(1) equals sim_run(1).  Errors as cue_step. */
int cone_step(cue_sim *sim, int32_t nsteps);

/* Advance cones and field together nsteps times: the coupled model of
 * Sec. 3.5 (cone step, Eq. 6-7) and Sec. 5.2 (field step) as above; at each
 * step the cones read C^n and the field becomes C^{n+1}.  Requires the cone
 * and field counters to be equal (else CUE_ERR_STATE); advances both.  The
 * library picks the kernel (CUE_OPT_PATH); every path gives the same values
 * bit for bit.  Errors as cue_step. */
int sim_run(cue_sim *sim, int32_t nsteps);

/*
 * sim_adjoint: gradients of the endpoint loss
 *     L = (1/n_axons) sum_a |p_a(T) - t_a|^2,   T = current step + nsteps,
 * with respect to D, lambda, the per-step source emissions e_k and the rate
 * map M (dL/dM_i; pass d_gmap = NULL to skip).  Needs a run without stopping:
 * cone_params.wall_mode = 1 (clamp) and stop_radius <= 0 (else CUE_ERR_ARG),
 * because stopping is a discrete event without a derivative.
 *
 * The call runs the coupled model nsteps forward from the handle's state,
 * keeping (C, p, d) every ckpt_every steps and storing every state of the last
 * segment, computes L, then walks back: each earlier segment is recomputed
 * from its checkpoint storing every step, and the adjoint field
 * mu = dL/dC^n is advanced backwards with the (symmetric) field operator while
 * the cone adjoint -- back through the clamp, the step length, the
 * normalisation Jacobians and the multilinear gradient sample -- scatters into
 * it.  With ckpt_every >= nsteps the whole run is stored once (nsteps + 1
 * states in the workspace) and nothing is recomputed: a workspace-for-time
 * trade the caller makes through ckpt_every.  Parameter gradients: dL/dD = dt/h^2 sum_n <mu^{n+1}, lap C^n>,
 * dL/dlambda = -dt sum_n <mu^{n+1}, C^n>, dL/de_k = sum_n mu^{n+1}[cell_k],
 * dL/dM = dt sum_n mu^{n+1}.
 *
 *   d_targets : dim*n_axons floats (SoA, like pos)
 *   d_adj_ws  : >= cue_adjoint_workspace_bytes(...) bytes, 256-byte aligned,
 *               caller-owned (checkpoints, one recomputed segment, adjoint
 *               state)
 *   outputs   : d_gD, d_glambda, d_loss one float each; d_gsrc n_src floats;
 *               d_gmap nx*ny(*nz) floats or NULL
 * On return (asynchronously) the handle is at step + nsteps, as after
 * sim_run(nsteps).  Errors: CUE_ERR_ARG, CUE_ERR_STATE, CUE_ERR_WORKSPACE,
 * CUE_ERR_CUDA.  Derivation: the model of the calls above (Sec. 3.5, 5.2);
 * the paper itself computes no gradients.
 */
int sim_adjoint(cue_sim *sim, const float *d_targets, int32_t nsteps, int32_t ckpt_every, void *d_adj_ws,
                size_t adj_ws_bytes, float *d_gD, float *d_glambda, float *d_gsrc, float *d_gmap, float *d_loss);

/* The endpoint loss L = (1/n_axons) sum_a |p_a - t_a|^2 of the handle's
 * current cone positions (the loss sim_adjoint differentiates), written to
 * d_loss (one float) on the handle's stream.  d_targets: dim*n_axons floats,
 * SoA like pos.  Errors: CUE_ERR_ARG, CUE_ERR_CUDA. */
int cue_endpoint_loss(cue_sim *sim, const float *d_targets, float *d_loss);

/* Change the field physics of a handle: the diffusion coefficient D and the
 * decay rate lambda of the field step (Sec. 5.2 grid model; Sec. 4.3 gives
 * each cue its own diffusion rate).  Takes effect at the next step; the cone
 * parameters, steering rule, buffers and counters stay.  Errors: CUE_ERR_ARG
 * (non-finite or negative values), CUE_ERR_UNSTABLE (D dt / h^2 > 1/(2 dim)
 * or lambda dt > 1; the handle is left unchanged). */
int cue_set_physics(cue_sim *sim, float D, float lambda);

/*
 * cue_adjoint_trace: a diagnostic hook for checking the backward pass on its
 * own.  With non-NULL buffers, every later sim_adjoint call on this handle
 * also copies out the FP32 forward states its backward pass reads (the states
 * recomputed from each checkpoint, exactly as the backward kernels see them):
 *   d_fields : >= (nsteps + 1) * cells floats; state n at d_fields + n*cells
 *   d_cones  : >= (nsteps + 1) * 2 * dim * n_axons floats; state n holds
 *              pos^n then dir^n (each SoA, as d_pos) at
 *              d_cones + n * 2 * dim * n_axons
 * for n = 0..nsteps relative to the call's first step.  max_states is the
 * number of states the buffers hold; a sim_adjoint call with
 * nsteps + 1 > max_states returns CUE_ERR_ARG.  Both NULL turns the trace off.
 * The buffers are the caller's.  The copies are queued on the handle's stream.
 * Errors: CUE_ERR_ARG (one buffer NULL, max_states < 2).
 */
int cue_adjoint_trace(cue_sim *sim, float *d_fields, float *d_cones, int64_t max_states);

/* Bytes of adjoint workspace sim_adjoint needs (0 for invalid arguments). */
size_t cue_adjoint_workspace_bytes(const cue_params *params, int32_t n_src, int32_t n_axons, int32_t nsteps,
                                   int32_t ckpt_every);

/* Step counters and the index (0 = d_field_a, 1 = d_field_b) of the buffer
 * that holds the current field. */
int cue_get_state(const cue_sim *sim, int64_t *field_step, int64_t *cone_step_out,
                  int32_t *cur_buffer);

/* Restore counters and the current-buffer index (for snapshots/resume). */
int cue_set_state(cue_sim *sim, int64_t field_step, int64_t cone_step_in, int32_t cur_buffer);

/* Re-target the stream used by later calls. */
int cue_set_stream(cue_sim *sim, void *stream);

/* Steering rule of the handle's cones: NULL = vector addition of the current
 * direction, the normalised cue gradient and noise (Sec. 3.5, Eq. 6-7; the
 * default); non-NULL = the SNR turn rule above (2D only).  Takes effect at the
 * next cone step.  The fused path and sim_adjoint support vector addition
 * only (the fused path is then skipped; sim_adjoint returns CUE_ERR_ARG).
 * Errors: CUE_ERR_ARG (3D handle, kd <= 0, non-finite values, c_min > c_max). */
int cue_set_steering(cue_sim *s, const cue_snr_params *snr);

/* Set an option (CUE_OPT_*). */
int cue_set_option(cue_sim *sim, int32_t option, int64_t value);

/* Read an option (CUE_OPT_*) or an informational value (CUE_INFO_*). */
int cue_get_option(const cue_sim *sim, int32_t option, int64_t *value);

/* Number of kernels this handle has launched so far. */
uint64_t cue_launch_count(const cue_sim *sim);

/* With CUE_OPT_TIME_KERNEL on: synchronise the stream and return the summed
 * device time (ms, from CUDA events on the handle's stream) and the number of
 * launches of the dominant field kernel (the fused kernel on the fused path,
 * the field stencil on the plain path, the one launch per call of the
 * persistent and resident paths) since the previous call; resets both. */
int cue_kernel_time(cue_sim *sim, double *total_ms, uint64_t *launches);

/* Synchronise the stream and return the number of cone updates (active
 * cone x step pairs) performed since the previous call; resets the count. */
int cue_cone_updates(cue_sim *sim, uint64_t *count);

/* Synchronise the stream, then return and clear the device status word:
 * CUE_OK, CUE_ERR_NONFINITE, CUE_ERR_BOUNDS, CUE_ERR_TIMEOUT or CUE_ERR_CUDA. */
int cue_status(cue_sim *sim);

/* Free the handle (never the caller's buffers).  NULL is accepted. */
void cue_destroy(cue_sim *sim);

/*
 * sim_run_static: the coupled run (as sim_run) for callers that cannot
 * allocate device memory -- code that runs under another framework's
 * allocator, a host that forbids cudaMalloc once it has started, or a caller
 * that must not grow the process's device footprint per call.  The paper has
 * no counterpart: this is an interface for such callers, not part of the
 * model.
 *
 * Arguments are those of cue_init (minus the workspace) plus the starting
 * step index step0 (both counters) and nsteps.  The fields, sources and cone
 * buffers are the caller's, as with cue_init; d_field_a holds C at step0 and
 * *cur_buffer_out receives the index of the buffer holding the result
 * (0 = d_field_a, 1 = d_field_b).  Work is queued on `stream`; the call
 * returns without synchronising.
 *
 * Scratch: one file-scope device array of cue_static_scratch_bytes()
 * (4 MiB), held by every GPU that loads the library until the process exits.
 * Problems needing more (cue_workspace_bytes) are rejected with
 * CUE_ERR_SCRATCH before anything is queued.  No cudaMalloc, cudaFree or
 * allocating library routine is called.  Every call looks up the array's
 * device address in the current context (cudaGetSymbolAddress); the first
 * lookup on a device loads the module there, so make the first call on a
 * device before any stream capture.  All calls on a device share the array
 * and it keeps the last call's contents (the parts that must start at zero,
 * the status word among them, are cleared by each call); calls whose GPU work
 * overlaps in time race on it.  Device-side problems (non-finite values,
 * skipped sources, a bounded wait that ran out) are recorded in the array's
 * status word: read it with cue_static_status after the call and before the
 * next one, which clears it.
 */
int sim_run_static(const cue_params *params, const cone_params *cone, float *d_field_a, float *d_field_b,
                   const int32_t *d_src_cell, const float *d_src_emit, int32_t n_src, const float *d_src_map,
                   float *d_pos, float *d_dir, uint8_t *d_active, int32_t n_axons, int64_t step0, int32_t nsteps,
                   void *stream, int32_t *cur_buffer_out);

/* Size in bytes of sim_run_static's device scratch array. */
size_t cue_static_scratch_bytes(void);

/* Status of the last sim_run_static call on the current device: synchronises
 * `stream` (the stream that call was given), then returns and clears the
 * status word of the fixed scratch array: CUE_OK, CUE_ERR_NONFINITE,
 * CUE_ERR_TIMEOUT, CUE_ERR_BOUNDS or CUE_ERR_CUDA.  Allocates nothing.  Like
 * sim_run_static it has no counterpart in the paper. */
int cue_static_status(void *stream);

/* Static description of a status code. */
const char *cue_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* CUE_H */
