// cue_api.cu -- the C ABI of libcue.so (declared in include/cue.h): argument
// checking, the handle, step bookkeeping and dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "cue_internal.h"

namespace cue {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

WorkspaceLayout workspace_layout(const cue_params &p, int n_src, int n_axons)
{
    WorkspaceLayout w;
    size_t off = 0;
    w.status_off = off;
    off += 256;
    w.src_xyz_off = off;
    off += align256(sizeof(float) * 3 * (size_t)(n_src > 0 ? n_src : 0));
    w.n_tiles = fused_tile_count(p);
    Fused3Geom g3;
    if (p.dim == 3 && fused3d_geometry(p, g3)) w.n_tiles = g3.boxes;   // the blocked 3D path's boxes
    const size_t nt = (size_t)(w.n_tiles > 0 ? w.n_tiles : 1);
    const size_t na = (size_t)(n_axons > 0 ? n_axons : 1);
    w.bin_count_off = off;
    off += align256(sizeof(int32_t) * 2 * nt);
    w.bin_ctl_off = off;
    off += 256;
    w.bin_cap = kFusedBinCap;
    if (w.n_tiles > 0 && (size_t)n_axons > (size_t)kFusedBinCap &&
        sizeof(int32_t) * 2 * nt * (size_t)n_axons <= kFusedBinBudget)
        w.bin_cap = n_axons;
    w.bin_list_off = off;
    off += align256(sizeof(int32_t) * 2 * nt * (w.n_tiles > 0 ? (size_t)w.bin_cap : 1));
    w.spill_off = off;
    off += align256(sizeof(int2) * 2 * (w.n_tiles > 0 ? na : 1));
    w.persist_off = off;
    if (p.dim == 2 && p.nx >= 4) {
        w.persist_items_cap = (size_t)persist_tiles(p.nx, p.ny, 1) + (na + kPersistConeChunk - 1) / kPersistConeChunk;
        off += 256 + align256(2 * sizeof(PInst)) + align256(sizeof(PItem) * w.persist_items_cap);
        const size_t ns = (size_t)(n_src > 0 ? n_src : 0);
        w.persist_src_off = off;
        off += align256(sizeof(PSrc) * ns) + align256(sizeof(int) * ns);
    }
    if (p.dim == 3 && fused3d_geometry(p, g3)) {     // the blocked 3D path's copy of its intermediate step
        w.inter_off = off;
        off += align256(sizeof(float) * (size_t)p.nx * p.ny * p.nz);
    }
    w.total = off;
    return w;
}

static constexpr size_t kEventRing = 512;

static void timing_collect(Sim &s, size_t slot)
{
    float ms = 0.f;
    if (cudaEventSynchronize(s.ev_stop[slot]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, s.ev_start[slot], s.ev_stop[slot]) == cudaSuccess) {
        s.timed_ms += ms;
        s.timed_launches++;
    }
}

void timing_begin(Sim &s)
{
    s.timing_now = false;
    if (!s.time_kernel) return;
    if (s.time_seen++ % s.time_period != 0) return;
    s.timing_now = true;
    if (s.ev_start.empty()) {
        s.ev_start.resize(kEventRing);
        s.ev_stop.resize(kEventRing);
        for (size_t i = 0; i < kEventRing; ++i) {
            cudaEventCreate(&s.ev_start[i]);
            cudaEventCreate(&s.ev_stop[i]);
        }
    }
    if (s.ev_live == kEventRing) {          // reuse the oldest pair: fold its time in first
        timing_collect(s, s.ev_next);
        s.ev_live--;
    }
    cudaEventRecord(s.ev_start[s.ev_next], s.stream);
}

void timing_end(Sim &s)
{
    if (!s.time_kernel || !s.timing_now) return;
    s.timing_now = false;
    cudaEventRecord(s.ev_stop[s.ev_next], s.stream);
    s.ev_next = (s.ev_next + 1) % kEventRing;
    s.ev_live++;
}

static void timing_drain(Sim &s)
{
    size_t first = (s.ev_next + kEventRing - s.ev_live) % kEventRing;
    for (size_t i = 0; i < s.ev_live; ++i) timing_collect(s, (first + i) % kEventRing);
    s.ev_live = 0;
}

static void timing_free(Sim &s)
{
    for (size_t i = 0; i < s.ev_start.size(); ++i) {
        cudaEventDestroy(s.ev_start[i]);
        cudaEventDestroy(s.ev_stop[i]);
    }
    s.ev_start.clear();
    s.ev_stop.clear();
}

static int sm_count_api()
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

int run_coupled(Sim &s, int nsteps)
{
    s.fused_used = false;
    s.persist_used = false;
    s.resident_used = false;
    s.cluster_used = false;
    // AUTO: the temporally blocked kernel when the grid gives every SM a tile;
    // else a cluster of CTAs with the grid in their distributed shared memory
    // where its measured step is the shortest (cluster_preferred); else one
    // block with the grid in shared memory; else the persistent launch (larger
    // small grids, or many cones); else plain.
    const bool small = !fused_supported(s) || fused_tile_count(s.params) < sm_count_api();
    int rc = 1;
    if (s.path == CUE_PATH_CLUSTER || (s.path == CUE_PATH_AUTO && small && cluster_preferred(s)))
        rc = run_cluster_if_supported(s, nsteps);
    if (rc != 1) return rc;
    if (s.path == CUE_PATH_RESIDENT || (s.path == CUE_PATH_AUTO && small)) rc = run_resident_if_supported(s, nsteps);
    if (rc != 1) return rc;
    if (s.path == CUE_PATH_PERSIST || (s.path == CUE_PATH_AUTO && small)) rc = run_persist_if_supported(s, nsteps);
    if (rc != 1) return rc;
    rc = run_fused3d_if_supported(s, nsteps, true);
    if (rc != 1) return rc;
    rc = run_fused_if_supported(s, nsteps);
    if (rc != 1) return rc;       // handled (0 = ok, < 0 = error)
    // 3D with the TMA field kernel: cones, field and sources of a step in one launch
    const bool merged3 = s.fd.dim == 3 && s.vec4 && field3d_tma_prepare(s);
    for (int k = 0; k < nsteps; ++k) {
        float *in = s.field[s.cur], *out = s.field[s.cur ^ 1];
        cudaError_t e;
        if (merged3) {
            bool cones = false, sources = false;
            timing_begin(s);
            e = launch_field3d_tma(s, s.cur, out, &cones, &sources);
            timing_end(s);
            s.launches++;
            // what the launch did not take: the cones read `in`, which no launch of this step writes
            if (e == cudaSuccess && !cones) e = launch_cone_step(s, in, (uint32_t)s.cone_step);
            if (e == cudaSuccess && !sources) e = launch_sources(s, out);
        } else {
            e = launch_cone_step(s, in, (uint32_t)s.cone_step);
            if (e == cudaSuccess) e = launch_field_and_sources(s, in, out);
        }
        if (e != cudaSuccess) return CUE_ERR_CUDA;
        s.cur ^= 1;
        s.field_step++;
        s.cone_step++;
    }
    return CUE_OK;
}

}  // namespace cue

using namespace cue;

struct cue_sim : public cue::Sim {};

namespace cue {

void sim_no_host_alloc(cue_sim *h)
{
    if (h) h->adapt_helpers = false;
}

int make_descs(const cue_params &params, const cone_params &cone, FieldDesc &f, ConeDesc &c)
{
    const int dim = params.dim;
    const float alpha = params.D * params.dt / (params.h * params.h);
    const float decay = params.lambda * params.dt;
    if (alpha > 1.0f / (2.0f * dim) * (1.0f + 1e-6f) || decay > 1.0f) return CUE_ERR_UNSTABLE;
    f.dim = dim;
    f.nx = params.nx;
    f.ny = params.ny;
    f.nz = dim == 3 ? params.nz : 1;
    f.h = params.h;
    f.alpha = alpha;
    f.decay = decay;
    f.dt = params.dt;
    f.beta = (float)(1.0 - 2.0 * dim * (double)alpha - (double)decay);
    f.inv_h = 1.0f / params.h;
    c.w_prev = cone.w_prev;
    c.w_grad = cone.w_grad;
    c.w_noise = cone.w_noise;
    c.step_len = cone.step_len;
    c.stop_r2 = cone.stop_radius > 0.f ? cone.stop_radius * cone.stop_radius : -1.0f;
    c.eps2 = cone.grad_eps * cone.grad_eps;
    c.inv2h = 1.0f / (2.0f * params.h);
    c.hi0 = (float)(f.nx - 1) * f.h;
    c.hi1 = (float)(f.ny - 1) * f.h;
    c.hi2 = (float)(f.nz - 1) * f.h;
    c.wall_mode = cone.wall_mode;
    c.key0 = (uint32_t)(cone.seed & 0xFFFFFFFFull);
    c.key1 = (uint32_t)(cone.seed >> 32);
    c.steer = 0;                     // vector addition until cue_set_steering says otherwise
    c.snr_gain = c.snr_width = c.snr_inv_kd = c.snr_cmin = c.snr_cmax = 0.0f;
    c.turn_c = 1.0f;
    c.turn_s = 0.0f;
    return CUE_OK;
}

bool params_ok(const cue_params *p)
{
    if (!p) return false;
    if (p->dim != 2 && p->dim != 3) return false;
    if (p->nx < 2 || p->ny < 2 || (p->dim == 3 && p->nz < 2)) return false;
    long long n = (long long)p->nx * p->ny * (p->dim == 3 ? p->nz : 1);
    if (n > (1LL << 31) - 1) return false;
    if (!(p->h > 0.f) || !(p->dt > 0.f) || !(p->D >= 0.f) || !(p->lambda >= 0.f)) return false;
    if (!std::isfinite(p->h) || !std::isfinite(p->dt) || !std::isfinite(p->D) || !std::isfinite(p->lambda))
        return false;
    if (p->boundary != 0) return false;
    return true;
}

bool cone_ok(const cone_params *c)
{
    if (!c) return false;
    if (c->wall_mode != 0 && c->wall_mode != 1) return false;
    if (c->reserved != 0) return false;
    const float v[] = {c->w_prev, c->w_grad, c->w_noise, c->step_len, c->stop_radius, c->grad_eps};
    for (float x : v)
        if (!std::isfinite(x)) return false;
    if (c->step_len < 0.f || c->grad_eps < 0.f) return false;
    return true;
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? CUE_OK : CUE_ERR_CUDA; }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace cue

extern "C" {

size_t cue_workspace_bytes(const cue_params *params, int32_t n_src, int32_t n_axons)
{
    if (!params_ok(params) || n_src < 0 || n_axons < 0) return 0;
    return workspace_layout(*params, n_src, n_axons).total;
}

int cue_init(cue_sim **out, const cue_params *params, const cone_params *cone, float *d_field_a,
             float *d_field_b, const int32_t *d_src_cell, const float *d_src_emit, int32_t n_src,
             const float *d_src_map, float *d_pos, float *d_dir, uint8_t *d_active, int32_t n_axons,
             void *d_workspace, size_t ws_bytes, void *stream)
{
    if (!out) return CUE_ERR_ARG;
    *out = nullptr;
    if (!params_ok(params) || !cone_ok(cone)) return CUE_ERR_ARG;
    if (!d_field_a || !d_field_b || d_field_a == d_field_b) return CUE_ERR_ARG;
    if (n_src < 0 || n_axons < 0) return CUE_ERR_ARG;
    if (n_src > 0 && (!d_src_cell || !d_src_emit)) return CUE_ERR_ARG;
    if (n_axons > 0 && (!d_pos || !d_dir || !d_active)) return CUE_ERR_ARG;
    const int dim = params->dim;
    FieldDesc fdesc;
    ConeDesc cdesc;
    if (make_descs(*params, *cone, fdesc, cdesc) != CUE_OK) return CUE_ERR_UNSTABLE;
    WorkspaceLayout wl = workspace_layout(*params, n_src, n_axons);
    if (!d_workspace || ws_bytes < wl.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return CUE_ERR_WORKSPACE;

    cue_sim *s = new (std::nothrow) cue_sim();
    if (!s) return CUE_ERR_ARG;
    s->params = *params;
    if (dim == 2) s->params.nz = 1;
    s->cone = *cone;
    s->fd = fdesc;
    s->cd = cdesc;
    const FieldDesc &f = s->fd;
    s->field[0] = d_field_a;
    s->field[1] = d_field_b;
    s->src_cell = d_src_cell;
    s->src_emit = d_src_emit;
    s->n_src = n_src;
    s->src_map = d_src_map;
    s->pos = d_pos;
    s->dir = d_dir;
    s->active = d_active;
    s->n_axons = n_axons;
    s->ws = static_cast<unsigned char *>(d_workspace);
    s->ws_bytes = ws_bytes;
    s->wl = wl;
    s->stream = static_cast<cudaStream_t>(stream);
    s->vec4 = (f.nx % 4 == 0) && aligned16(d_field_a) && aligned16(d_field_b) &&
              (!d_src_map || aligned16(d_src_map));
    cudaError_t e = cudaMemsetAsync(s->ws, 0, 256, s->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->ws + wl.bin_count_off, 0, wl.bin_list_off - wl.bin_count_off, s->stream);

    if (e == cudaSuccess) e = launch_src_xyz(*s);
    if (e != cudaSuccess) {
        delete s;
        return CUE_ERR_CUDA;
    }
    *out = s;
    return CUE_OK;
}

int cue_step(cue_sim *s, int32_t nsteps)
{
    if (!s || nsteps < 0) return CUE_ERR_ARG;
    if (s->field_step + nsteps > 0xFFFFFFFFLL) return CUE_ERR_STATE;
    s->fused_used = false;
    int rc = run_fused3d_if_supported(*s, nsteps, false);
    if (rc != 1) return rc;
    rc = field_fused_if_supported(*s, nsteps);
    if (rc != 1) return rc;
    s->fused_used = false;
    for (int k = 0; k < nsteps; ++k) {
        float *in = s->field[s->cur], *out = s->field[s->cur ^ 1];
        cudaError_t e = launch_field_and_sources(*s, in, out);
        if (e != cudaSuccess) return CUE_ERR_CUDA;
        s->cur ^= 1;
        s->field_step++;
    }
    return CUE_OK;
}

int cone_step(cue_sim *s, int32_t nsteps)
{
    if (!s || nsteps < 0) return CUE_ERR_ARG;
    if (s->cone_step + nsteps > 0xFFFFFFFFLL) return CUE_ERR_STATE;
    for (int k = 0; k < nsteps; ++k) {
        cudaError_t e = launch_cone_step(*s, s->field[s->cur], (uint32_t)s->cone_step);
        if (e != cudaSuccess) return CUE_ERR_CUDA;
        s->cone_step++;
    }
    return CUE_OK;
}

int sim_run(cue_sim *s, int32_t nsteps)
{
    if (!s || nsteps < 0) return CUE_ERR_ARG;
    if (s->cone_step != s->field_step) return CUE_ERR_STATE;
    if (s->field_step + nsteps > 0xFFFFFFFFLL) return CUE_ERR_STATE;
    return run_coupled(*s, nsteps);
}

size_t cue_adjoint_workspace_bytes(const cue_params *params, int32_t n_src, int32_t n_axons, int32_t nsteps,
                                   int32_t ckpt_every)
{
    if (!params_ok(params) || n_src < 0 || n_axons < 0) return 0;
    cue_params p = *params;
    if (p.dim == 2) p.nz = 1;
    return adjoint_workspace_bytes(p, n_src, n_axons, nsteps, ckpt_every);
}

int sim_adjoint(cue_sim *s, const float *d_targets, int32_t nsteps, int32_t ckpt_every, void *d_adj_ws,
                size_t adj_ws_bytes, float *d_gD, float *d_glambda, float *d_gsrc, float *d_gmap, float *d_loss)
{
    if (!s || nsteps <= 0 || ckpt_every <= 0) return CUE_ERR_ARG;
    if (!d_gD || !d_glambda || !d_loss || (s->n_src > 0 && !d_gsrc) || (s->n_axons > 0 && !d_targets))
        return CUE_ERR_ARG;
    if (s->cone.wall_mode != 1 || s->cd.stop_r2 >= 0.0f) return CUE_ERR_ARG;   // needs a run without stopping
    if (s->cd.steer != 0) return CUE_ERR_ARG;                                    // vector addition only
    if (s->cone_step != s->field_step) return CUE_ERR_STATE;
    if (s->field_step + nsteps > 0xFFFFFFFFLL) return CUE_ERR_STATE;
    if (s->adj_trace_field && (int64_t)nsteps + 1 > s->adj_trace_cap) return CUE_ERR_ARG;
    return run_adjoint(*s, d_targets, nsteps, ckpt_every, d_adj_ws, adj_ws_bytes, d_gD, d_glambda, d_gsrc, d_gmap,
                       d_loss);
}

int cue_endpoint_loss(cue_sim *s, const float *d_targets, float *d_loss)
{
    if (!s || !d_loss || (s->n_axons > 0 && !d_targets)) return CUE_ERR_ARG;
    return cuda_err(launch_endpoint_loss(*s, d_targets, d_loss));
}

int cue_set_physics(cue_sim *s, float D, float lambda)
{
    if (!s || !std::isfinite(D) || !std::isfinite(lambda) || D < 0.0f || lambda < 0.0f) return CUE_ERR_ARG;
    cue_params p = s->params;
    p.D = D;
    p.lambda = lambda;
    FieldDesc f;
    ConeDesc c;
    const int rc = make_descs(p, s->cone, f, c);
    if (rc != CUE_OK) return rc;
    s->params = p;
    s->fd = f;                   // the cone descriptor (and its steering rule) stays
    s->persist_ready = false;    // the persistent path's instance record holds the field descriptor
    return CUE_OK;
}

int cue_adjoint_trace(cue_sim *s, float *d_fields, float *d_cones, int64_t max_states)
{
    if (!s) return CUE_ERR_ARG;
    if (!d_fields && !d_cones) {
        s->adj_trace_field = nullptr;
        s->adj_trace_cone = nullptr;
        s->adj_trace_cap = 0;
        return CUE_OK;
    }
    if (!d_fields || !d_cones || max_states < 2) return CUE_ERR_ARG;
    s->adj_trace_field = d_fields;
    s->adj_trace_cone = d_cones;
    s->adj_trace_cap = max_states;
    return CUE_OK;
}

int cue_get_state(const cue_sim *s, int64_t *field_step, int64_t *cone_step_out, int32_t *cur_buffer)
{
    if (!s) return CUE_ERR_ARG;
    if (field_step) *field_step = s->field_step;
    if (cone_step_out) *cone_step_out = s->cone_step;
    if (cur_buffer) *cur_buffer = s->cur;
    return CUE_OK;
}

int cue_set_state(cue_sim *s, int64_t field_step, int64_t cone_step_in, int32_t cur_buffer)
{
    if (!s || field_step < 0 || cone_step_in < 0 || field_step > 0xFFFFFFFFLL ||
        cone_step_in > 0xFFFFFFFFLL || (cur_buffer != 0 && cur_buffer != 1))
        return CUE_ERR_ARG;
    s->field_step = field_step;
    s->cone_step = cone_step_in;
    s->cur = cur_buffer;
    return CUE_OK;
}

int cue_set_stream(cue_sim *s, void *stream)
{
    if (!s) return CUE_ERR_ARG;
    s->stream = static_cast<cudaStream_t>(stream);
    return CUE_OK;
}

int cue_set_steering(cue_sim *s, const cue_snr_params *snr)
{
    if (!s) return CUE_ERR_ARG;
    if (!snr) {
        s->cd.steer = 0;
        s->persist_ready = false;
        return CUE_OK;
    }
    if (s->fd.dim != 2) return CUE_ERR_ARG;
    const float v[] = {snr->gain, snr->width, snr->kd, snr->c_min, snr->turn};
    for (float x : v)
        if (!std::isfinite(x)) return CUE_ERR_ARG;
    if (!(snr->kd > 0.0f) || std::isnan(snr->c_max) || snr->c_min > snr->c_max) return CUE_ERR_ARG;
    s->cd.steer = 1;
    s->cd.snr_gain = snr->gain;
    s->cd.snr_width = snr->width;
    s->cd.snr_inv_kd = (float)(1.0 / (double)snr->kd);
    s->cd.snr_cmin = snr->c_min;
    s->cd.snr_cmax = snr->c_max;
    s->cd.turn_c = (float)std::cos((double)snr->turn);
    s->cd.turn_s = (float)std::sin((double)snr->turn);
    s->persist_ready = false;          // the persistent path's instance record holds the cone parameters
    if (s->path == CUE_PATH_FUSED) s->path = CUE_PATH_AUTO;
    return CUE_OK;
}

int cue_set_option(cue_sim *s, int32_t option, int64_t value)
{
    if (!s) return CUE_ERR_ARG;
    switch (option) {
    case CUE_OPT_PATH:
        if (value != CUE_PATH_AUTO && value != CUE_PATH_PLAIN && value != CUE_PATH_FUSED &&
            value != CUE_PATH_PERSIST && value != CUE_PATH_RESIDENT && value != CUE_PATH_CLUSTER)
            return CUE_ERR_ARG;
        if (value == CUE_PATH_CLUSTER && !cluster_supported(*s)) return CUE_ERR_ARG;
        if (value == CUE_PATH_FUSED && !fused_supported(*s) && !fused3d_supported(*s)) return CUE_ERR_ARG;
        if (value == CUE_PATH_PERSIST && !persist_supported(*s)) return CUE_ERR_ARG;
        if (value == CUE_PATH_RESIDENT && !resident_supported(*s)) return CUE_ERR_ARG;
        s->path = (int)value;
        return CUE_OK;
    case CUE_OPT_PERSIST_ROWS:
        if (value != 0 && value != 1 && value != 2 && value != 4) return CUE_ERR_ARG;
        s->persist_rows = (int)value;
        return CUE_OK;
    case CUE_OPT_PERSIST_BLOCKS:
        if (value < 0 || value > 8) return CUE_ERR_ARG;
        s->persist_bpsm = (int)value;
        return CUE_OK;
    case CUE_OPT_WAIT_LIMIT:
        if (value < 0 || value > (1LL << 40)) return CUE_ERR_ARG;
        s->persist_limit = value;
        return CUE_OK;
    case CUE_OPT_BARRIER_PHANTOM:
        if (value < 0 || value > 1024) return CUE_ERR_ARG;
        s->persist_phantom = (int)value;
        return CUE_OK;
    case CUE_OPT_CLUSTER_CTAS: {
        if (value != 0 && value != kClusterSize && value != kClusterSizeLarge) return CUE_ERR_ARG;
        const int old = s->cluster_opt;
        s->cluster_opt = (int)value;
        s->cluster_pick = -1;
        if (s->path == CUE_PATH_CLUSTER && !cluster_supported(*s)) {   // keep the selected path runnable
            s->cluster_opt = old;
            s->cluster_pick = -1;
            return CUE_ERR_ARG;
        }
        return CUE_OK;
    }
    case CUE_OPT_TEMPORAL_DEPTH:
        if (value < 0 || value > kMaxTemporalDepth) return CUE_ERR_ARG;
        s->temporal_depth = (int)value;
        s->geom_ready = false;
        return CUE_OK;
    case CUE_OPT_ROWS_PER_THREAD:
        if (value < 0 || value > 64) return CUE_ERR_ARG;
        s->rows_per_thread = (int)value;
        return CUE_OK;
    case CUE_OPT_TIME_KERNEL:
        if (value < 0 || value > 1 << 20) return CUE_ERR_ARG;
        if (!value && s->time_kernel) timing_drain(*s);
        s->time_kernel = value != 0;
        s->time_period = value > 0 ? (int)value : 1;
        s->time_seen = 0;
        return CUE_OK;
    default:
        return CUE_ERR_ARG;
    }
}

int cue_kernel_time(cue_sim *s, double *total_ms, uint64_t *launches)
{
    if (!s) return CUE_ERR_ARG;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return CUE_ERR_CUDA;
    timing_drain(*s);
    if (total_ms) *total_ms = s->timed_ms;
    if (launches) *launches = s->timed_launches;
    s->timed_ms = 0.0;
    s->timed_launches = 0;
    return CUE_OK;
}

int cue_get_option(const cue_sim *s, int32_t option, int64_t *value)
{
    if (!s || !value) return CUE_ERR_ARG;
    switch (option) {
    case CUE_OPT_PATH: *value = s->path; return CUE_OK;
    case CUE_OPT_TEMPORAL_DEPTH: *value = s->temporal_depth; return CUE_OK;
    case CUE_OPT_ROWS_PER_THREAD: *value = s->rows_per_thread; return CUE_OK;
    case CUE_OPT_TIME_KERNEL: *value = s->time_kernel ? s->time_period : 0; return CUE_OK;
    case CUE_INFO_LAST_PATH:
        *value = s->fused_used      ? CUE_PATH_FUSED
                 : s->persist_used  ? CUE_PATH_PERSIST
                 : s->resident_used ? CUE_PATH_RESIDENT
                 : s->cluster_used  ? CUE_PATH_CLUSTER
                                    : CUE_PATH_PLAIN;
        return CUE_OK;
    case CUE_OPT_PERSIST_ROWS: *value = s->persist_rows; return CUE_OK;
    case CUE_OPT_PERSIST_BLOCKS: *value = s->persist_bpsm; return CUE_OK;
    case CUE_OPT_WAIT_LIMIT: *value = s->persist_limit; return CUE_OK;
    case CUE_OPT_BARRIER_PHANTOM: *value = s->persist_phantom; return CUE_OK;
    case CUE_OPT_CLUSTER_CTAS: *value = s->cluster_opt; return CUE_OK;
    case CUE_INFO_GRID: *value = s->cluster_used ? s->cluster_last : s->persist_grid; return CUE_OK;
    case CUE_INFO_HELPERS: *value = s->help_last; return CUE_OK;
    case CUE_INFO_TILE:
        if (s->fd.dim == 3) *value = s->geom3_ready ? (int64_t)128 | ((int64_t)s->geom3.TY << 16) : 0;
        else *value = s->geom_ready ? (int64_t)s->geom.TX | ((int64_t)s->geom.TY << 16) : 0;
        return CUE_OK;
    case CUE_INFO_DEPTH:
        if (s->fd.dim == 3) *value = s->geom3_ready ? 2 : 0;
        else *value = s->geom_ready ? s->geom.K : 0;
        return CUE_OK;
    default: return CUE_ERR_ARG;
    }
}

uint64_t cue_launch_count(const cue_sim *s) { return s ? s->launches : 0; }

int cue_cone_updates(cue_sim *s, uint64_t *count)
{
    if (!s || !count) return CUE_ERR_ARG;
    unsigned long long v = 0;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return CUE_ERR_CUDA;
    if (cudaMemcpy(&v, s->cone_counter(), sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return CUE_ERR_CUDA;
    if (cudaMemset(s->cone_counter(), 0, sizeof(v)) != cudaSuccess) return CUE_ERR_CUDA;
    *count = v;
    return CUE_OK;
}

int cue_status(cue_sim *s)
{
    if (!s) return CUE_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return CUE_ERR_CUDA;
    unsigned word = 0;
    e = cudaMemcpy(&word, s->status(), sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return CUE_ERR_CUDA;
    if (word) {
        e = cudaMemset(s->status(), 0, sizeof(unsigned));
        if (e != cudaSuccess) return CUE_ERR_CUDA;
    }
    if (word & kStatusNonFinite) return CUE_ERR_NONFINITE;
    if (word & kStatusTimeout) return CUE_ERR_TIMEOUT;
    if (word & kStatusBounds) return CUE_ERR_BOUNDS;
    e = cudaGetLastError();
    return cuda_err(e);
}

void cue_destroy(cue_sim *s)
{
    if (!s) return;
    if (!s->ev_start.empty()) {
        cudaStreamSynchronize(s->stream);
        timing_free(*s);
    }
    if (s->help_ev) {
        cudaEventSynchronize(s->help_ev);       // the readback lands before its word goes
        cudaEventDestroy(s->help_ev);
    }
    if (s->help_host) cudaFreeHost(s->help_host);
    delete s;
}

const char *cue_strerror(int code)
{
    switch (code) {
    case CUE_OK: return "ok";
    case CUE_ERR_ARG: return "invalid argument";
    case CUE_ERR_UNSTABLE: return "unstable parameters: D dt / h^2 > 1/(2 dim) or lambda dt > 1";
    case CUE_ERR_CUDA: return "CUDA runtime error";
    case CUE_ERR_NONFINITE: return "non-finite value produced on the device";
    case CUE_ERR_TIMEOUT: return "bounded device-side wait timed out";
    case CUE_ERR_BOUNDS: return "source cell index outside the grid (skipped)";
    case CUE_ERR_WORKSPACE: return "workspace missing, too small or not 256-byte aligned";
    case CUE_ERR_STATE: return "call order violated (cone and field step counters differ)";
    case CUE_ERR_SCRATCH: return "problem needs more scratch than sim_run_static's fixed 4 MiB device array";
    default: return "unknown status code";
    }
}

}  // extern "C"
