/*
 * cue_oracle.c -- plain FP64 CPU oracle for the guidance-cue field and the
 * growth-cone step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the model that the CUDA path is checked against.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * build, load or call it; the product library never links it, and it shares
 * no code, header, table or constant with the CUDA sources.
 *
 * The model (Mihut, Morgan & Kaiser, "GPU Simulation of Axon Growth and
 * Guidance through Cue Diffusion"):
 *   - the cue lives on a fixed Eulerian grid (Sec. 5.2), diffuses at a
 *     per-cue rate and is emitted by sources placed pseudo-randomly
 *     (Sec. 4.3); its influence falls off with distance from the source
 *     (Sec. 3.5, "Diffusion of guidance molecules").  Written as an explicit
 *     update  C' = C + dt (D lap(C) - lambda C) + S  on nodes x = i h with
 *     no-flux walls;
 *   - each growth cone advances a fixed distance per step along its
 *     direction, which is steered by vector addition of the current
 *     direction and the cue direction it senses across its width
 *     (Sec. 3.5, "Growth cone steering mechanisms", Eq. 6-7), plus a
 *     Gaussian term (Sec. 3.5, the N(SNR,1) decision) drawn from a
 *     stateless per-thread counter-based generator (Sec. 5.1) through the
 *     Box-Muller transform (Sec. 3.2, normal-deviate method);
 *   - a cone stops when it leaves the simulation bounds (Sec. 3.4) or, when
 *     enabled, when it comes within a radius of a cue source, tested on
 *     squared distances (Sec. 3.3).
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   - nodes at x = i h, domain [0,(N-1)h] per axis;
 *   - no-flux wall = a missing neighbour contributes no flux term
 *     (equivalently a ghost node equal to the edge node);
 *   - the per-step emission e_k is added to the source node after the
 *     stencil, unscaled by dt; a dense rate map M enters as dt*M;
 *   - cones and field both read the state of step n;
 *   - node gradient = central difference with ghost = edge; the gradient at
 *     a point is the bilinear (2D) / trilinear (3D) interpolation of the node
 *     gradients;
 *   - ghat = g/|g| if |g|^2 > eps^2 else 0; v = w_p d + w_g ghat + w_n xi;
 *     d' = v/|v| unless |v|^2 <= 1e-30 (then d' = d); p' = p + l d';
 *   - noise: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *     key = (seed lo, seed hi), counter = (axon, step, 0, 0); uniforms
 *     u1 = ((x0>>8)+1) 2^-24 in (0,1], u2 = (x1>>8) 2^-24 in [0,1), and the
 *     same for (x2, x3); Box-Muller gives xi0, xi1 from (u1,u2), xi2 from
 *     (u3,u4);
 *   - wall mode 0 (stop): if p' leaves the domain the cone becomes inactive
 *     and keeps p, d of step n; wall mode 1 (clamp): each coordinate of p' is
 *     clamped to the domain and d' is kept;
 *   - source stop: after the move, inactive if |p' - x_k|^2 <= r^2 for some
 *     source node x_k.
 *
 * Pins (tests that do not re-type this code): hand-enumerated single steps,
 * exact mass conservation, the exact FTCS variance growth, the heat kernel,
 * the pure-decay closed form, the DCT-II steady-state solve, mirror and
 * transpose symmetry, self-adjointness of the no-flux Laplacian, exact
 * gradients of linear and quadratic fields, the scalar heading recurrence,
 * straight lines, the normal law of the noise, and Philox against an
 * independent implementation.  Whole-run trajectories (hundreds of coupled
 * steps) are parity unpinned by design: they are chaotic with respect to
 * rounding and are compared only as endpoint statistics.
 *
 * Layout: fields are dense row-major arrays with x fastest,
 * index = i + nx (j + ny k).  Cone state is structure-of-arrays:
 * pos[c*n + a] is coordinate c of cone a (same for dir).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int dim;            /* 2 or 3 */
    int nx, ny, nz;     /* nodes per axis (nz = 1 in 2D) */
    double h, D, lambda, dt;
} orc_grid;

typedef struct {
    double w_prev, w_grad, w_noise, step_len;
    double stop_radius; /* <= 0: off */
    double grad_eps;
    int wall_mode;      /* 0 = stop at the wall, 1 = clamp to the wall */
    uint64_t seed;
    /* steering rule: 0 = vector addition of the current direction and the
     * sensed cue direction (Sec. 3.5, Eq. 6-7); 1 = the SNR turn rule of
     * Sec. 3.5, Eq. 5 (2D): the cone turns by snr_turn to the right when a draw
     * from N(SNR, 1) is positive, else to the left, while the cue value at the
     * cone lies in [snr_cmin, snr_cmax]; outside that window it keeps its
     * direction. */
    int steer;
    double snr_gain;    /* the gain of Eq. 5 */
    double snr_width;   /* growth-cone width w: gradient steepness mu = w |grad C| / C */
    double snr_kd;      /* concentration scale: gamma = C / kd */
    double snr_cmin, snr_cmax;
    double snr_turn;    /* turn angle per step (the paper: pi/30) */
} orc_cone;

static int64_t nodes_of(const orc_grid *g)
{
    return (int64_t)g->nx * g->ny * (g->dim == 3 ? g->nz : 1);
}

static int extent(const orc_grid *g, int axis)
{
    return axis == 0 ? g->nx : axis == 1 ? g->ny : g->nz;
}

/* ------------------------------------------------------------------------
 * Philox-4x32-10, written from the SC'11 definition: each round multiplies
 * counter words 0 and 2 by the two round constants, forms the 64-bit
 * products' high and low halves, and mixes the high halves with the other
 * two words and the round key; the key is bumped by the two Weyl constants
 * between rounds.
 * ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1]: the top 24 bits plus one, times 2^-24. */
static double unit_open0(uint32_t x) { return ((double)(x >> 8) + 1.0) * (1.0 / 16777216.0); }
/* Uniform in [0,1): the top 24 bits times 2^-24. */
static double unit_open1(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* Gaussian noise vector of cone `axon` at step `step` (Box-Muller on the
 * four Philox words); xi[0..dim-1] are i.i.d. N(0,1). */
void orc_noise(uint64_t seed, uint32_t axon, uint32_t step, int dim, double xi[3])
{
    const double two_pi = 6.283185307179586476925286766559;
    uint32_t ctr[4] = {axon, step, 0u, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u1 = unit_open0(x[0]), u2 = unit_open1(x[1]);
    double r = sqrt(-2.0 * log(u1));
    xi[0] = r * cos(two_pi * u2);
    xi[1] = r * sin(two_pi * u2);
    xi[2] = 0.0;
    if (dim == 3) {
        double u3 = unit_open0(x[2]), u4 = unit_open1(x[3]);
        double r2 = sqrt(-2.0 * log(u3));
        xi[2] = r2 * cos(two_pi * u4);
    }
}

void orc_noise_many(uint64_t seed, int n, const uint32_t *axon, const uint32_t *step,
                    int dim, double *xi /* [n][3] */)
{
    for (int a = 0; a < n; ++a)
        orc_noise(seed, axon[a], step[a], dim, xi + 3 * (size_t)a);
}

void orc_philox_many(int n, const uint32_t *ctr /* [n][4] */, const uint32_t *key /* [n][2] */,
                     uint32_t *out /* [n][4] */)
{
    for (int a = 0; a < n; ++a)
        orc_philox4x32_10(ctr + 4 * (size_t)a, key + 2 * (size_t)a, out + 4 * (size_t)a);
}

/* ------------------------------------------------------------------------
 * Field: one explicit step.  For every node, each existing axis neighbour j
 * contributes alpha (C_j - C_i); missing neighbours (walls) contribute
 * nothing; decay removes lambda dt C_i.  Then the point sources add their
 * per-step emission, then a dense rate map adds dt M_i.
 * ---------------------------------------------------------------------- */
/* Threads of the node loop below (rows are independent, so any count gives
 * the same result bit for bit); 1 unless the timed baseline asks for more,
 * and only where the library was built with OpenMP. */
static int orc_nthreads = 1;

void orc_set_threads(int n) { orc_nthreads = n > 0 ? n : 1; }

int orc_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

void orc_field_step(const orc_grid *g, const double *C, double *Cn,
                    const int32_t *src_cell, const double *src_emit, int n_src,
                    const double *src_map)
{
    const double alpha = g->D * g->dt / (g->h * g->h);
    const double decay = g->lambda * g->dt;
    const int nx = g->nx, ny = g->ny, nz = (g->dim == 3) ? g->nz : 1;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static) num_threads(orc_nthreads) if (orc_nthreads > 1)
#endif
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t c = i * sx + j * sy + k * sz;
                double ci = C[c];
                double flux = 0.0;
                if (i > 0)      flux += C[c - sx] - ci;
                if (i < nx - 1) flux += C[c + sx] - ci;
                if (j > 0)      flux += C[c - sy] - ci;
                if (j < ny - 1) flux += C[c + sy] - ci;
                if (g->dim == 3) {
                    if (k > 0)      flux += C[c - sz] - ci;
                    if (k < nz - 1) flux += C[c + sz] - ci;
                }
                Cn[c] = ci + alpha * flux - decay * ci;
            }
    for (int s = 0; s < n_src; ++s)
        Cn[src_cell[s]] += src_emit[s];
    if (src_map) {
        int64_t n = nodes_of(g);
        for (int64_t c = 0; c < n; ++c)
            Cn[c] += g->dt * src_map[c];
    }
}

/* ------------------------------------------------------------------------
 * The same field step on a window of a grid too large to hold in the oracle:
 * `Wp` holds the input values of the window grown by one node on every side
 * ((wx + 2) x (wy + 2) x (wz + 2) values, x fastest; entries outside the grid
 * are never read), the window's first node is (ox, oy, oz) in global
 * coordinates, and `out` receives C' of the wx x wy x wz window nodes.  Walls
 * are decided by global coordinates; the point sources whose node lies in the
 * window are added, as in orc_field_step (no rate map).
 * ---------------------------------------------------------------------- */
void orc_field_window(const orc_grid *g, const double *Wp, int64_t ox, int64_t oy, int64_t oz, int wx, int wy,
                      int wz, const int64_t *src_cell, const double *src_emit, int n_src, double *out)
{
    const double alpha = g->D * g->dt / (g->h * g->h);
    const double decay = g->lambda * g->dt;
    const int64_t nx = g->nx, ny = g->ny, nz = (g->dim == 3) ? g->nz : 1;
    const int64_t px = wx + 2, py = wy + 2;          /* padded window extents */
    const int64_t sx = 1, sy = px, sz = px * py;
    const int pz0 = (g->dim == 3) ? 1 : 0;           /* 2D windows have no z padding */
    for (int k = 0; k < wz; ++k)
        for (int j = 0; j < wy; ++j)
            for (int i = 0; i < wx; ++i) {
                const int64_t gi = ox + i, gj = oy + j, gk = oz + k;
                const int64_t c = (i + 1) * sx + (j + 1) * sy + (k + pz0) * sz;
                double ci = Wp[c];
                double flux = 0.0;
                if (gi > 0)      flux += Wp[c - sx] - ci;
                if (gi < nx - 1) flux += Wp[c + sx] - ci;
                if (gj > 0)      flux += Wp[c - sy] - ci;
                if (gj < ny - 1) flux += Wp[c + sy] - ci;
                if (g->dim == 3) {
                    if (gk > 0)      flux += Wp[c - sz] - ci;
                    if (gk < nz - 1) flux += Wp[c + sz] - ci;
                }
                out[i + (int64_t)wx * (j + (int64_t)wy * k)] = ci + alpha * flux - decay * ci;
            }
    for (int s = 0; s < n_src; ++s) {
        const int64_t cell = src_cell[s];
        const int64_t gi = cell % nx, gj = (cell / nx) % ny, gk = cell / (nx * ny);
        if (gi >= ox && gi < ox + wx && gj >= oy && gj < oy + wy && gk >= oz && gk < oz + wz)
            out[(gi - ox) + (int64_t)wx * ((gj - oy) + (int64_t)wy * (gk - oz))] += src_emit[s];
    }
}

/* ------------------------------------------------------------------------
 * Gradient.  Node gradient: central differences, a missing neighbour
 * replaced by the node itself (ghost = edge), so on a wall node the
 * one-sided difference is halved.  Point gradient: bilinear / trilinear
 * interpolation of the node gradients of the cell that holds p, the cell's
 * lower corner clamped to [0, N-2] on each axis.
 * ---------------------------------------------------------------------- */
static double node_value(const orc_grid *g, const double *C, int i, int j, int k)
{
    return C[(int64_t)i + (int64_t)g->nx * ((int64_t)j + (int64_t)g->ny * k)];
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

void orc_node_gradient(const orc_grid *g, const double *C, int i, int j, int k, double out[3])
{
    const double inv2h = 1.0 / (2.0 * g->h);
    int nz = (g->dim == 3) ? g->nz : 1;
    out[0] = (node_value(g, C, clampi(i + 1, 0, g->nx - 1), j, k) -
              node_value(g, C, clampi(i - 1, 0, g->nx - 1), j, k)) * inv2h;
    out[1] = (node_value(g, C, i, clampi(j + 1, 0, g->ny - 1), k) -
              node_value(g, C, i, clampi(j - 1, 0, g->ny - 1), k)) * inv2h;
    out[2] = 0.0;
    if (g->dim == 3)
        out[2] = (node_value(g, C, i, j, clampi(k + 1, 0, nz - 1)) -
                  node_value(g, C, i, j, clampi(k - 1, 0, nz - 1))) * inv2h;
}

void orc_gradient_at(const orc_grid *g, const double *C, const double p[3], double out[3])
{
    int lo[3] = {0, 0, 0};
    double f[3] = {0.0, 0.0, 0.0};
    for (int ax = 0; ax < g->dim; ++ax) {
        double s = p[ax] / g->h;
        int i0 = (int)floor(s);
        i0 = clampi(i0, 0, extent(g, ax) - 2);
        lo[ax] = i0;
        f[ax] = s - (double)i0;
    }
    out[0] = out[1] = out[2] = 0.0;
    int kcorners = (g->dim == 3) ? 2 : 1;
    for (int dk = 0; dk < kcorners; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                double w = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]);
                if (g->dim == 3) w *= (dk ? f[2] : 1.0 - f[2]);
                double gn[3];
                orc_node_gradient(g, C, lo[0] + di, lo[1] + dj, lo[2] + dk, gn);
                out[0] += w * gn[0];
                out[1] += w * gn[1];
                out[2] += w * gn[2];
            }
}

/* Cue value at p (2D): bilinear interpolation of the four nodes of the cell
 * holding p, the cell chosen as for the gradient. */
double orc_value_at(const orc_grid *g, const double *C, const double p[3])
{
    int lo[2];
    double f[2];
    for (int ax = 0; ax < 2; ++ax) {
        double s = p[ax] / g->h;
        int i0 = (int)floor(s);
        i0 = clampi(i0, 0, extent(g, ax) - 2);
        lo[ax] = i0;
        f[ax] = s - (double)i0;
    }
    double v = 0.0;
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
            double w = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]);
            v += w * C[(int64_t)(lo[0] + di) + (int64_t)g->nx * (lo[1] + dj)];
        }
    return v;
}

/* SNR of the cone's gradient measurement (Sec. 3.5, Eq. 5, 2D):
 *   SNR = gain * mu * sqrt(gamma / (1 + gamma)^3) * sin(theta - theta_NGF),
 * gamma = C/kd (background concentration), mu = w |grad C| / C (gradient
 * steepness across the cone), theta the heading and theta_NGF the gradient's
 * direction, sin(theta - theta_NGF) from the cross product of the unit vectors
 * (d_y g_x - d_x g_y) / |g| as in the Eq. 6-7 discussion. */
double orc_snr(const orc_cone *cp, double Cp, const double *gr, const double *d)
{
    double gn = sqrt(gr[0] * gr[0] + gr[1] * gr[1]);
    if (!(gn > 0.0) || !(Cp > 0.0)) return 0.0;
    double gamma = Cp / cp->snr_kd;
    double mu = cp->snr_width * gn / Cp;
    double sin_rel = (d[1] * gr[0] - d[0] * gr[1]) / gn;
    double onep = 1.0 + gamma;
    return cp->snr_gain * mu * sqrt(gamma / (onep * onep * onep)) * sin_rel;
}

void orc_gradient_many(const orc_grid *g, const double *C, int n, const double *p /* [n][3] */,
                       double *out /* [n][3] */)
{
    for (int a = 0; a < n; ++a)
        orc_gradient_at(g, C, p + 3 * (size_t)a, out + 3 * (size_t)a);
}

/* ------------------------------------------------------------------------
 * Growth cones: one step of every active cone on the field C of this step.
 * pos/dir are SoA [dim][n]; active is 0/1.
 * ---------------------------------------------------------------------- */
void orc_cone_step(const orc_grid *g, const orc_cone *cp, const double *C, uint32_t step,
                   int n, double *pos, double *dir, uint8_t *active,
                   const int32_t *src_cell, int n_src)
{
    const int dim = g->dim;
    const double eps2 = cp->grad_eps * cp->grad_eps;
    const double r2 = cp->stop_radius * cp->stop_radius;
    for (int a = 0; a < n; ++a) {
        if (!active[a]) continue;
        double p[3] = {0, 0, 0}, d[3] = {0, 0, 0};
        for (int c = 0; c < dim; ++c) {
            p[c] = pos[(size_t)c * n + a];
            d[c] = dir[(size_t)c * n + a];
        }
        /* sensed cue direction */
        double gr[3];
        orc_gradient_at(g, C, p, gr);
        /* noise */
        double xi[3];
        orc_noise(cp->seed, (uint32_t)a, step, dim, xi);
        double dn[3] = {d[0], d[1], d[2]};
        if (cp->steer == 1 && dim == 2) {
            /* SNR rule (Eq. 5): inside the detectable window, turn right by the
             * turn angle when SNR + z > 0 (z = the cone's first normal draw: a
             * draw from N(SNR, 1) is SNR + z), else left */
            double Cp = orc_value_at(g, C, p);
            if (Cp >= cp->snr_cmin && Cp <= cp->snr_cmax) {
                double snr = orc_snr(cp, Cp, gr, d);
                double ang = (snr + xi[0] > 0.0) ? -cp->snr_turn : cp->snr_turn;
                double cs = cos(ang), sn = sin(ang);
                double r0 = d[0] * cs - d[1] * sn, r1 = d[0] * sn + d[1] * cs;
                double inv = 1.0 / sqrt(r0 * r0 + r1 * r1);
                dn[0] = r0 * inv;
                dn[1] = r1 * inv;
            }
        } else {
            double gn2 = 0.0;
            for (int c = 0; c < dim; ++c) gn2 += gr[c] * gr[c];
            double ghat[3] = {0, 0, 0};
            if (gn2 > eps2) {
                double inv = 1.0 / sqrt(gn2);
                for (int c = 0; c < dim; ++c) ghat[c] = gr[c] * inv;
            }
            /* vector addition of previous direction, cue direction and noise */
            double v[3] = {0, 0, 0}, vn2 = 0.0;
            for (int c = 0; c < dim; ++c) {
                v[c] = cp->w_prev * d[c] + cp->w_grad * ghat[c] + cp->w_noise * xi[c];
                vn2 += v[c] * v[c];
            }
            if (vn2 > 1e-30) {
                double inv = 1.0 / sqrt(vn2);
                for (int c = 0; c < dim; ++c) dn[c] = v[c] * inv;
            }
        }
        double pn[3] = {0, 0, 0};
        for (int c = 0; c < dim; ++c) pn[c] = p[c] + cp->step_len * dn[c];
        /* walls */
        int outside = 0;
        for (int c = 0; c < dim; ++c) {
            double hi = (extent(g, c) - 1) * g->h;
            if (pn[c] < 0.0 || pn[c] > hi) {
                outside = 1;
                if (cp->wall_mode == 1) pn[c] = pn[c] < 0.0 ? 0.0 : hi;
            }
        }
        if (outside && cp->wall_mode == 0) {
            active[a] = 0;          /* stays at p, d of this step */
            continue;
        }
        for (int c = 0; c < dim; ++c) {
            pos[(size_t)c * n + a] = pn[c];
            dir[(size_t)c * n + a] = dn[c];
        }
        /* source proximity, squared-distance test */
        if (cp->stop_radius > 0.0) {
            for (int s = 0; s < n_src; ++s) {
                int64_t cell = src_cell[s];
                double xs[3];
                xs[0] = (double)(cell % g->nx) * g->h;
                xs[1] = (double)((cell / g->nx) % g->ny) * g->h;
                xs[2] = (dim == 3) ? (double)(cell / ((int64_t)g->nx * g->ny)) * g->h : 0.0;
                double d2 = 0.0;
                for (int c = 0; c < dim; ++c) d2 += (pn[c] - xs[c]) * (pn[c] - xs[c]);
                if (d2 <= r2) { active[a] = 0; break; }
            }
        }
    }
}

/* ------------------------------------------------------------------------
 * nsteps of the coupled model starting at step `step0`: the cones step on
 * C^n, then the field advances to C^{n+1}.  C holds the field on entry and
 * exit; work is a scratch field of the same size.
 * ---------------------------------------------------------------------- */
void orc_run(const orc_grid *g, const orc_cone *cp, double *C, double *work,
             uint32_t step0, int nsteps,
             const int32_t *src_cell, const double *src_emit, int n_src, const double *src_map,
             int n, double *pos, double *dir, uint8_t *active)
{
    int64_t nn = nodes_of(g);
    for (int s = 0; s < nsteps; ++s) {
        uint32_t step = step0 + (uint32_t)s;
        if (n > 0)
            orc_cone_step(g, cp, C, step, n, pos, dir, active, src_cell, n_src);
        orc_field_step(g, C, work, src_cell, src_emit, n_src, src_map);
        memcpy(C, work, (size_t)nn * sizeof(double));
    }
}

/* ------------------------------------------------------------------------
 * Adjoint of the endpoint loss  L = (1/n) sum_a |p_a^T - t_a|^2  with respect
 * to D, lambda, the per-step emissions e_k and the rate map M, for the
 * no-stopping workload (wall mode 1 = clamp, no source stop).  The field does
 * not depend on the cones; the cones read C^n through the gradient sample.
 *
 * Forward, stored: C^n and (p^n, d^n) for n = 0..T.
 * Backward, n = T-1 .. 0, with pbar/dbar = dL/dp^{n+1}, dL/dd^{n+1} and
 * mu = dL/dC^{n+1} on entry:
 *   parameter terms of C^{n+1} = C^n + alpha lap(C^n) - lambda dt C^n + s:
 *     dL/dD      += (dt/h^2) <mu, lap(C^n)>
 *     dL/dlambda -= dt <mu, C^n>
 *     dL/de_k    += mu[cell_k]
 *     dL/dM_i    += dt mu_i
 *   field:  mu <- A mu   (A = I + alpha lap - lambda dt, symmetric)
 *   cones:  back through p' = clamp(p + l d'), d' = v/|v|,
 *           v = w_p d + w_g g/|g| + w_n xi, g = grad C^n (p); the sampled
 *           gradient is linear in C^n, so its adjoint adds into mu (now
 *           dL/dC^n), and bilinear in p, so it adds into pbar.
 * Written from the derivation above; pinned by central finite differences of
 * the forward loss (tests).
 * ---------------------------------------------------------------------- */
static void lap_apply(const orc_grid *g, const double *x, double *out)
{
    const int nx = g->nx, ny = g->ny, nz = (g->dim == 3) ? g->nz : 1;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t c = i + j * sy + k * sz;
                double xi = x[c], s = 0.0;
                if (i > 0) s += x[c - 1] - xi;
                if (i < nx - 1) s += x[c + 1] - xi;
                if (j > 0) s += x[c - sy] - xi;
                if (j < ny - 1) s += x[c + sy] - xi;
                if (g->dim == 3) {
                    if (k > 0) s += x[c - sz] - xi;
                    if (k < nz - 1) s += x[c + sz] - xi;
                }
                out[c] = s;
            }
}

/* Backward through one clamp-mode cone step of cone a (2D or 3D). */
static void cone_step_adjoint(const orc_grid *g, const orc_cone *cp, const double *C, uint32_t step,
                              uint32_t a, const double *p, const double *d, double *pbar, double *dbar,
                              double *mu)
{
    const int dim = g->dim;
    const double eps2 = cp->grad_eps * cp->grad_eps;
    /* recompute the forward step */
    int lo[3] = {0, 0, 0};
    double f[3] = {0, 0, 0};
    for (int ax = 0; ax < dim; ++ax) {
        double s = p[ax] / g->h;
        int i0 = (int)floor(s);
        i0 = clampi(i0, 0, extent(g, ax) - 2);
        lo[ax] = i0;
        f[ax] = s - (double)i0;
    }
    const int kc = (dim == 3) ? 2 : 1;
    double gn[8][3], w[8], dw[8][3];
    int corner[8][3];
    int nc = 0;
    double gr[3] = {0, 0, 0};
    for (int dk = 0; dk < kc; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                double wx = di ? f[0] : 1.0 - f[0], wy = dj ? f[1] : 1.0 - f[1];
                double wz = (dim == 3) ? (dk ? f[2] : 1.0 - f[2]) : 1.0;
                double sx = di ? 1.0 : -1.0, sy = dj ? 1.0 : -1.0, sz = dk ? 1.0 : -1.0;
                corner[nc][0] = lo[0] + di;
                corner[nc][1] = lo[1] + dj;
                corner[nc][2] = lo[2] + dk;
                orc_node_gradient(g, C, corner[nc][0], corner[nc][1], corner[nc][2], gn[nc]);
                w[nc] = wx * wy * wz;
                dw[nc][0] = sx * wy * wz / g->h;      /* d w / d p_x */
                dw[nc][1] = wx * sy * wz / g->h;
                dw[nc][2] = (dim == 3) ? wx * wy * sz / g->h : 0.0;
                for (int k = 0; k < 3; ++k) gr[k] += w[nc] * gn[nc][k];
                ++nc;
            }
    double gn2 = 0.0;
    for (int k = 0; k < dim; ++k) gn2 += gr[k] * gr[k];
    double gnorm = sqrt(gn2), ghat[3] = {0, 0, 0};
    int has_g = gn2 > eps2;
    if (has_g)
        for (int k = 0; k < dim; ++k) ghat[k] = gr[k] / gnorm;
    double xi[3];
    orc_noise(cp->seed, a, step, dim, xi);
    double v[3] = {0, 0, 0}, vn2 = 0.0;
    for (int k = 0; k < dim; ++k) {
        v[k] = cp->w_prev * d[k] + cp->w_grad * ghat[k] + cp->w_noise * xi[k];
        vn2 += v[k] * v[k];
    }
    double vn = sqrt(vn2), dn[3] = {d[0], d[1], d[2]};
    int has_v = vn2 > 1e-30;
    if (has_v)
        for (int k = 0; k < dim; ++k) dn[k] = v[k] / vn;
    double qbar[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
        double q = p[k] + cp->step_len * dn[k];
        double hi = (extent(g, k) - 1) * g->h;
        qbar[k] = (q < 0.0 || q > hi) ? 0.0 : pbar[k];
    }
    /* back through d' = v/|v| (or d' = d) */
    double dnbar[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) dnbar[k] = dbar[k] + cp->step_len * qbar[k];
    double vbar[3] = {0, 0, 0}, dbar_out[3] = {0, 0, 0};
    if (has_v) {
        double dot = 0.0;
        for (int k = 0; k < dim; ++k) dot += dn[k] * dnbar[k];
        for (int k = 0; k < dim; ++k) vbar[k] = (dnbar[k] - dn[k] * dot) / vn;
        for (int k = 0; k < dim; ++k) dbar_out[k] = cp->w_prev * vbar[k];
    } else {
        for (int k = 0; k < dim; ++k) dbar_out[k] = dnbar[k];
    }
    /* back through ghat = g/|g| */
    double gbar[3] = {0, 0, 0};
    if (has_g) {
        double dot = 0.0;
        for (int k = 0; k < dim; ++k) dot += ghat[k] * cp->w_grad * vbar[k];
        for (int k = 0; k < dim; ++k) gbar[k] = (cp->w_grad * vbar[k] - ghat[k] * dot) / gnorm;
    }
    /* back through the sample: position (bilinear weights) and field (node differences) */
    double pbar_out[3] = {qbar[0], qbar[1], qbar[2]};
    const double inv2h = 1.0 / (2.0 * g->h);
    int nz = (dim == 3) ? g->nz : 1;
    for (int c = 0; c < nc; ++c) {
        for (int m = 0; m < dim; ++m)
            for (int k = 0; k < dim; ++k) pbar_out[m] += gbar[k] * dw[c][m] * gn[c][k];
        int i = corner[c][0], j = corner[c][1], kk = corner[c][2];
        for (int k = 0; k < dim; ++k) {
            double coef = gbar[k] * w[c] * inv2h;
            int ip[3] = {i, j, kk}, im[3] = {i, j, kk};
            int ext = extent(g, k);
            if (k == 2) ext = nz;
            ip[k] = clampi(ip[k] + 1, 0, ext - 1);
            im[k] = clampi(im[k] - 1, 0, ext - 1);
            mu[(int64_t)ip[0] + (int64_t)g->nx * ((int64_t)ip[1] + (int64_t)g->ny * ip[2])] += coef;
            mu[(int64_t)im[0] + (int64_t)g->nx * ((int64_t)im[1] + (int64_t)g->ny * im[2])] -= coef;
        }
    }
    for (int k = 0; k < 3; ++k) {
        pbar[k] = (k < dim) ? pbar_out[k] : 0.0;
        dbar[k] = (k < dim) ? dbar_out[k] : 0.0;
    }
}

/* The backward pass alone, over given forward states: Cs holds C^n (nodes
 * values each) and Ps / Ds hold p^n / d^n (SoA [dim][n] each) for
 * n = 0..T.  Returns the loss at p^T; writes dL/dD, dL/dlambda, dL/de_k
 * (n_src) and dL/dM (nodes).  `work` holds 3 * nodes doubles.  Fed the
 * states of the oracle's own forward run this is exactly orc_adjoint's
 * backward; fed another program's stored states it gives the derivative that
 * program's backward pass must produce from them (the same states in, so the
 * forward's rounding drops out of the comparison). */
double orc_adjoint_from_states(const orc_grid *g, const orc_cone *cp, const int32_t *src_cell, int n_src, int n,
                               const double *targets, int T, const double *Cs, const double *Ps,
                               const double *Ds, double *gD, double *glam, double *gsrc, double *gmap,
                               double *work)
{
    const int dim = g->dim;
    const int64_t nn = nodes_of(g);
    const size_t cs = (size_t)dim * n;
    double *mu = work, *mu2 = mu + nn, *lapC = mu2 + nn;
    /* loss and its adjoint at T */
    double loss = 0.0;
    const double *PT = Ps + (size_t)T * cs;
    double *pbar = (double *)malloc((cs + 1) * sizeof(double)), *dbar = (double *)malloc((cs + 1) * sizeof(double));
    for (int a = 0; a < n; ++a)
        for (int k = 0; k < dim; ++k) {
            double e = PT[(size_t)k * n + a] - targets[(size_t)k * n + a];
            loss += e * e;
            pbar[(size_t)k * n + a] = 2.0 * e / n;
            dbar[(size_t)k * n + a] = 0.0;
        }
    if (n > 0) loss /= n;
    const double alpha_dD = g->dt / (g->h * g->h);
    *gD = 0.0;
    *glam = 0.0;
    for (int s = 0; s < n_src; ++s) gsrc[s] = 0.0;
    for (int64_t c = 0; c < nn; ++c) gmap[c] = 0.0;
    for (int64_t c = 0; c < nn; ++c) mu[c] = 0.0;          /* dL/dC^T = 0 */
    const double alpha = g->D * g->dt / (g->h * g->h), decay = g->lambda * g->dt;
    for (int s = T - 1; s >= 0; --s) {
        const double *Cn = Cs + (size_t)s * nn;
        /* parameter terms with mu = dL/dC^{s+1} */
        lap_apply(g, Cn, lapC);
        double sD = 0.0, sL = 0.0;
        for (int64_t c = 0; c < nn; ++c) {
            sD += mu[c] * lapC[c];
            sL += mu[c] * Cn[c];
            gmap[c] += g->dt * mu[c];
        }
        *gD += alpha_dD * sD;
        *glam -= g->dt * sL;
        for (int k = 0; k < n_src; ++k) gsrc[k] += mu[src_cell[k]];
        /* field: mu <- A mu */
        lap_apply(g, mu, mu2);
        for (int64_t c = 0; c < nn; ++c) mu2[c] = mu[c] + alpha * mu2[c] - decay * mu[c];
        memcpy(mu, mu2, (size_t)nn * sizeof(double));
        /* cones of step s: pbar/dbar from step s+1 to step s, and dL/dC^s */
        const double *P = Ps + (size_t)s * cs, *Dd = Ds + (size_t)s * cs;
        for (int a = 0; a < n; ++a) {
            double p[3] = {0, 0, 0}, d[3] = {0, 0, 0}, pb[3] = {0, 0, 0}, db[3] = {0, 0, 0};
            for (int k = 0; k < dim; ++k) {
                p[k] = P[(size_t)k * n + a];
                d[k] = Dd[(size_t)k * n + a];
                pb[k] = pbar[(size_t)k * n + a];
                db[k] = dbar[(size_t)k * n + a];
            }
            cone_step_adjoint(g, cp, Cn, (uint32_t)s, (uint32_t)a, p, d, pb, db, mu);
            for (int k = 0; k < dim; ++k) {
                pbar[(size_t)k * n + a] = pb[k];
                dbar[(size_t)k * n + a] = db[k];
            }
        }
    }
    free(pbar);
    free(dbar);
    return loss;
}

/* Forward T clamp-mode steps from (C0, pos0, dir0), then the adjoint.
 * Returns the loss; writes dL/dD, dL/dlambda, dL/de_k (n_src), dL/dM (cells).
 * pos0/dir0/targets are SoA [dim][n].  Memory: (T+1) fields and cone states.
 * state_binary32 != 0 stores every forward state (field, positions, directions) rounded to
 * binary32: a perturbation of exactly the size single-precision storage makes, used by the
 * tests to measure how strongly a case's gradients depend on it.  0 is the oracle proper.
 * The backward pass is orc_adjoint_from_states over the stored states. */
double orc_adjoint(const orc_grid *g, const orc_cone *cp, const double *C0,
                   const int32_t *src_cell, const double *src_emit, int n_src, const double *src_map,
                   int n, const double *pos0, const double *dir0, const double *targets, int T,
                   double *gD, double *glam, double *gsrc, double *gmap, double *Cs, double *Ps, double *Ds,
                   double *work, int state_binary32)
{
    const int dim = g->dim;
    const int64_t nn = nodes_of(g);
    const size_t cs = (size_t)dim * n;
    uint8_t *act = (uint8_t *)work;                  /* n bytes (all stay active) */
    double *mu = (double *)((uint8_t *)work + ((n + 15) / 16) * 16);
    /* forward, storing every state */
    memcpy(Cs, C0, (size_t)nn * sizeof(double));
    memcpy(Ps, pos0, cs * sizeof(double));
    memcpy(Ds, dir0, cs * sizeof(double));
    for (int a = 0; a < n; ++a) act[a] = 1;
    for (int s = 0; s < T; ++s) {
        memcpy(Ps + (size_t)(s + 1) * cs, Ps + (size_t)s * cs, cs * sizeof(double));
        memcpy(Ds + (size_t)(s + 1) * cs, Ds + (size_t)s * cs, cs * sizeof(double));
        orc_cone_step(g, cp, Cs + (size_t)s * nn, (uint32_t)s, n, Ps + (size_t)(s + 1) * cs,
                      Ds + (size_t)(s + 1) * cs, act, src_cell, n_src);
        orc_field_step(g, Cs + (size_t)s * nn, Cs + (size_t)(s + 1) * nn, src_cell, src_emit, n_src, src_map);
        if (state_binary32) {
            double *Cn = Cs + (size_t)(s + 1) * nn, *Pn = Ps + (size_t)(s + 1) * cs, *Dn = Ds + (size_t)(s + 1) * cs;
            for (int64_t i = 0; i < nn; ++i) Cn[i] = (double)(float)Cn[i];
            for (size_t i = 0; i < cs; ++i) {
                Pn[i] = (double)(float)Pn[i];
                Dn[i] = (double)(float)Dn[i];
            }
        }
    }
    return orc_adjoint_from_states(g, cp, src_cell, n_src, n, targets, T, Cs, Ps, Ds, gD, glam, gsrc, gmap, mu);
}

/* Loss of the forward run alone (for finite differences). */
double orc_endpoint_loss(const orc_grid *g, const orc_cone *cp, const double *C0,
                         const int32_t *src_cell, const double *src_emit, int n_src, const double *src_map,
                         int n, const double *pos0, const double *dir0, const double *targets, int T)
{
    const int dim = g->dim;
    const int64_t nn = nodes_of(g);
    double *C = (double *)malloc((size_t)nn * sizeof(double)), *W = (double *)malloc((size_t)nn * sizeof(double));
    double *P = (double *)malloc((size_t)dim * n * sizeof(double)), *D = (double *)malloc((size_t)dim * n * sizeof(double));
    uint8_t *act = (uint8_t *)malloc((size_t)n + 1);
    memcpy(C, C0, (size_t)nn * sizeof(double));
    memcpy(P, pos0, (size_t)dim * n * sizeof(double));
    memcpy(D, dir0, (size_t)dim * n * sizeof(double));
    for (int a = 0; a < n; ++a) act[a] = 1;
    orc_run(g, cp, C, W, 0, T, src_cell, src_emit, n_src, src_map, n, P, D, act);
    double loss = 0.0;
    for (int a = 0; a < n; ++a)
        for (int k = 0; k < dim; ++k) {
            double e = P[(size_t)k * n + a] - targets[(size_t)k * n + a];
            loss += e * e;
        }
    free(C); free(W); free(P); free(D); free(act);
    return loss / n;
}

/* ==========================================================================
 * Connectivity (the paper's collision-detection and graph stages).
 *
 * Uniform grid (Sec. 3.5, "Diffusion of guidance molecules"): each point's
 * cell is its linear grid index (the hash), the (cell, id) pairs are sorted,
 * and a change of cell id between consecutive sorted entries marks a cell's
 * start and end (Table 1).  Connection test (Sec. 3.3): a growth cone at x and
 * a neuron at y connect when |x - y|^2 < r^2, r the sum of the two radii (the
 * squared form avoids the square root).  Adjacency list (Sec. 3.4, Fig. 4):
 * vertex heads V_a into one edge array E_a, the edges of vertex i+1 after
 * those of i.  Traversal (Sec. 3.4, Fig. 5): breadth-first, level by level,
 * the level (cost) of each vertex from a source.
 * ========================================================================== */

/* Grid cell of one point: floor(x / cell) per axis, clamped into the grid. */
static int64_t grid_cell_of(int dim, const double *pos, int n, int i, double cell, const int32_t *grid)
{
    int64_t c = 0, stride = 1;
    for (int ax = 0; ax < dim; ++ax) {
        int64_t k = (int64_t)floor(pos[(size_t)ax * n + i] / cell);
        if (k < 0) k = 0;
        if (k > grid[ax] - 1) k = grid[ax] - 1;
        c += k * stride;
        stride *= grid[ax];
    }
    return c;
}

typedef struct {
    int64_t cell;
    int32_t id;
} cell_pair;

static int cmp_cell_pair(const void *a, const void *b)
{
    const cell_pair *x = (const cell_pair *)a, *y = (const cell_pair *)b;
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Hash, sort by (cell, id), cell start / one-past-end (-1 for empty cells). */
void orc_bin_points(int dim, int n, const double *pos, double cell, const int32_t *grid, int32_t *cell_of,
                    int32_t *sorted_id, int32_t *cell_start, int32_t *cell_end)
{
    int64_t ncell = 1;
    for (int ax = 0; ax < dim; ++ax) ncell *= grid[ax];
    for (int64_t c = 0; c < ncell; ++c) cell_start[c] = cell_end[c] = -1;
    cell_pair *pr = (cell_pair *)malloc(sizeof(cell_pair) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        pr[i].cell = grid_cell_of(dim, pos, n, i, cell, grid);
        pr[i].id = i;
        cell_of[i] = (int32_t)pr[i].cell;
    }
    qsort(pr, (size_t)n, sizeof(cell_pair), cmp_cell_pair);
    for (int j = 0; j < n; ++j) {
        sorted_id[j] = pr[j].id;
        if (j == 0 || pr[j].cell != pr[j - 1].cell) cell_start[pr[j].cell] = j;
        if (j == n - 1 || pr[j].cell != pr[j + 1].cell) cell_end[pr[j].cell] = j + 1;
    }
    free(pr);
}

/* Every (active cone, neuron) pair with |x - y|^2 < radius^2, except a cone and
 * its own neuron, as (owner[cone], neuron), cones in order then neurons in
 * order; at most cap pairs are written, the full count is returned. */
int orc_connect(int dim, int n_cones, const double *pos, const int32_t *owner, const uint8_t *active,
                int n_neurons, const double *npos, double radius, int cap, int32_t *src, int32_t *dst)
{
    const double r2 = radius * radius;
    int count = 0;
    for (int a = 0; a < n_cones; ++a) {
        if (active && !active[a]) continue;
        for (int j = 0; j < n_neurons; ++j) {
            if (owner[a] == j) continue;
            double d2 = 0.0;
            for (int ax = 0; ax < dim; ++ax) {
                double e = pos[(size_t)ax * n_cones + a] - npos[(size_t)ax * n_neurons + j];
                d2 += e * e;
            }
            if (d2 < r2) {
                if (count < cap) {
                    src[count] = owner[a];
                    dst[count] = j;
                }
                ++count;
            }
        }
    }
    return count;
}

typedef struct {
    int32_t s, d;
} edge_pair;

static int cmp_edge(const void *a, const void *b)
{
    const edge_pair *x = (const edge_pair *)a, *y = (const edge_pair *)b;
    if (x->s != y->s) return (x->s > y->s) - (x->s < y->s);
    return (x->d > y->d) - (x->d < y->d);
}

/* Adjacency list of the distinct edges: row[v] .. row[v+1] index col, sorted. */
int orc_csr(int nv, int ne, const int32_t *src, const int32_t *dst, int32_t *row, int32_t *col)
{
    edge_pair *e = (edge_pair *)malloc(sizeof(edge_pair) * (size_t)(ne > 0 ? ne : 1));
    for (int k = 0; k < ne; ++k) {
        e[k].s = src[k];
        e[k].d = dst[k];
    }
    qsort(e, (size_t)ne, sizeof(edge_pair), cmp_edge);
    int m = 0;
    for (int k = 0; k < ne; ++k)
        if (k == 0 || e[k].s != e[k - 1].s || e[k].d != e[k - 1].d) e[m++] = e[k];
    for (int v = 0; v <= nv; ++v) row[v] = 0;
    for (int k = 0; k < m; ++k) row[e[k].s + 1]++;
    for (int v = 0; v < nv; ++v) row[v + 1] += row[v];
    for (int k = 0; k < m; ++k) col[k] = e[k].d;
    free(e);
    return m;
}

/* Breadth-first levels from `source` (-1: unreachable), a FIFO queue. */
void orc_bfs(int nv, const int32_t *row, const int32_t *col, int source, int32_t *level)
{
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    for (int v = 0; v < nv; ++v) level[v] = -1;
    int head = 0, tail = 0;
    if (source >= 0 && source < nv) {
        level[source] = 0;
        q[tail++] = source;
    }
    while (head < tail) {
        int v = q[head++];
        for (int k = row[v]; k < row[v + 1]; ++k) {
            int u = col[k];
            if (level[u] < 0) {
                level[u] = level[v] + 1;
                q[tail++] = u;
            }
        }
    }
    free(q);
}
