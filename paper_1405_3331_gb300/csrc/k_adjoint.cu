// k_adjoint.cu -- gradients of the endpoint loss L = (1/n) sum_a |p_a^T - t_a|^2
// with respect to D, lambda, the per-step source emissions e_k and the rate
// map M, for runs without stopping (wall clamp, no source stop).
//
// The field does not depend on the cones; cone a reads C^n through the
// sampled gradient at step n.  With mu = dL/dC^{n+1} and (pbar, dbar) =
// dL/d(p, d)^{n+1}, going backwards through step n:
//   dL/dD      += (dt/h^2) <lap(mu), C^n>      (lap is symmetric)
//   dL/dlambda -= dt <mu, C^n>
//   dL/de_k    += mu[cell_k];   dL/dM += dt mu
//   mu <- A mu                  (A = I + alpha lap - lambda dt: the forward stencil)
//   cones: back through p' = clamp(p + l d'), d' = v/|v|, v = w_p d + w_g g/|g|
//          + w_n xi, g = bilinear/trilinear gradient of C^n at p; the gradient is
//          linear in C^n (its adjoint scatters into mu, now dL/dC^n) and
//          multilinear in p (adds into pbar).
// Memory: the forward keeps (C, p, d) every ckpt_every steps; each segment is
// recomputed with the plain kernels, storing every step, then walked
// backwards (two kernels per step).
#include <algorithm>

#include "cue_internal.h"

namespace cue {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

// Block sum of two doubles, added once per block to acc[0], acc[1].
__device__ __forceinline__ void block_add2(double a, double b, double *acc)
{
    __shared__ double sa[32], sb[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) / 32;
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
        if (lane == 0) {
            atomicAdd(&acc[0], a);
            atomicAdd(&acc[1], b);
        }
    }
}

// mu_out = A mu_in;  acc[0] += <lap(mu_in), C>;  acc[1] += <mu_in, C>;  S += mu_in.
// The adjoint field is carried in FP64: cones near the diffusion front, where
// |grad C| is tiny, inject contributions of order 1/|grad C| that cancel in
// these sums, and FP32 would lose them.
__global__ void __launch_bounds__(256) adj_field_kernel(FieldDesc f, const double *__restrict__ mu_in,
                                                        double *__restrict__ mu_out, const float *__restrict__ C,
                                                        double *S, double *acc)
{
    const size_t n = (size_t)f.nx * f.ny * f.nz;
    const size_t sy = f.nx, sz = (size_t)f.nx * f.ny;
    const double alpha = f.alpha, beta = f.beta;
    double tD = 0.0, tL = 0.0;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % f.nx);
        const int j = (int)((c / f.nx) % f.ny);
        const int k = (int)(c / sz);
        const double m = mu_in[c];
        const double xm = i > 0 ? mu_in[c - 1] : m;
        const double xp = i < f.nx - 1 ? mu_in[c + 1] : m;
        const double ym = j > 0 ? mu_in[c - sy] : m;
        const double yp = j < f.ny - 1 ? mu_in[c + sy] : m;
        double sum = (xm + xp) + (ym + yp), nn = 4.0;
        if (f.dim == 3) {
            const double zm = k > 0 ? mu_in[c - sz] : m;
            const double zp = k < f.nz - 1 ? mu_in[c + sz] : m;
            sum += zm + zp;
            nn = 6.0;
        }
        const double cc = C[c];
        tD = fma(sum - nn * m, cc, tD);
        tL = fma(m, cc, tL);
        if (S) S[c] += m;
        mu_out[c] = fma(alpha, sum, beta * m);
    }
    block_add2(tD, tL, acc);
}

// Node (i,j,k) as a linear index.
__device__ __forceinline__ size_t node_index(const FieldDesc &f, int i, int j, int k)
{
    return (size_t)i + (size_t)f.nx * ((size_t)j + (size_t)f.ny * k);
}

// Backward through one clamp-mode cone step.  p, d: state at step n;
// pbar, dbar: in dL/d(p,d)^{n+1}, out dL/d(p,d)^n; the field part is scattered
// into mu (atomic adds).
template <int DIM>
__device__ __forceinline__ void cone_adjoint(const FieldDesc &f, const ConeDesc &c, const float *__restrict__ C,
                                             uint32_t axon, uint32_t step, const float *p, const float *d,
                                             float *pbar, float *dbar, double *mu)
{
    const size_t sy = f.nx, sz = (size_t)f.nx * f.ny;
    auto ld = [&](int i, int j, int k) { return __ldg(C + (size_t)i + sy * j + sz * k); };
    // forward recomputation with the forward's own functions (same decisions)
    float g[DIM];
    sample_gradient<DIM>(f, c, p, ld, g);
    float gn2 = 0.f;
#pragma unroll
    for (int i = 0; i < DIM; ++i) gn2 = fmaf(g[i], g[i], gn2);
    const bool has_g = gn2 > c.eps2;
    const float ginv = has_g ? rsqrtf(gn2) : 0.0f;
    float xi[DIM];
    cone_noise<DIM>(c.key0, c.key1, axon, step, xi);
    float v[DIM], vn2 = 0.f, ghat[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        ghat[i] = g[i] * ginv;
        v[i] = c.w_prev * d[i] + c.w_grad * ghat[i] + c.w_noise * xi[i];
        vn2 = fmaf(v[i], v[i], vn2);
    }
    const bool has_v = vn2 > 1e-30f;
    const float vinv = has_v ? rsqrtf(vn2) : 0.0f;
    float dn[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) dn[i] = has_v ? v[i] * vinv : d[i];
    const float hi[3] = {c.hi0, c.hi1, c.hi2};
    // adjoint
    float qbar[DIM], dnbar[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        const float q = fmaf(c.step_len, dn[i], p[i]);
        qbar[i] = (q < 0.0f || q > hi[i]) ? 0.0f : pbar[i];
        dnbar[i] = fmaf(c.step_len, qbar[i], dbar[i]);
    }
    float vbar[DIM];
    if (has_v) {
        float dot = 0.f;
#pragma unroll
        for (int i = 0; i < DIM; ++i) dot = fmaf(dn[i], dnbar[i], dot);
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            vbar[i] = (dnbar[i] - dn[i] * dot) * vinv;
            dbar[i] = c.w_prev * vbar[i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            vbar[i] = 0.f;
            dbar[i] = dnbar[i];
        }
    }
    float gbar[DIM];
    {
        float dot = 0.f;
#pragma unroll
        for (int i = 0; i < DIM; ++i) dot = fmaf(ghat[i], c.w_grad * vbar[i], dot);
#pragma unroll
        for (int i = 0; i < DIM; ++i) gbar[i] = has_g ? (c.w_grad * vbar[i] - ghat[i] * dot) * ginv : 0.0f;
    }
    // back through the sample: bilinear / trilinear weights (position) and the
    // node central differences (field)
    int lo[3] = {0, 0, 0};
    float fr[3] = {0.f, 0.f, 0.f};
    cell_of<DIM>(f, p, lo, fr);
    const int ext[3] = {f.nx, f.ny, f.nz};
    float pb[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) pb[i] = qbar[i];
    const int kc = DIM == 3 ? 2 : 1;
    for (int e = 0; e < kc; ++e)
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int idx[3] = {lo[0] + a, lo[1] + b, lo[2] + e};
                const float w1[3] = {a ? fr[0] : 1.0f - fr[0], b ? fr[1] : 1.0f - fr[1],
                                     DIM == 3 ? (e ? fr[2] : 1.0f - fr[2]) : 1.0f};
                const float sg[3] = {a ? 1.0f : -1.0f, b ? 1.0f : -1.0f, e ? 1.0f : -1.0f};
                const float w = w1[0] * w1[1] * w1[2];
                // node gradient at this corner (ghost = edge) and the scatter of gbar
                float gnode[DIM];
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    int ip[3] = {idx[0], idx[1], idx[2]}, im[3] = {idx[0], idx[1], idx[2]};
                    ip[k] = min(ip[k] + 1, ext[k] - 1);
                    im[k] = max(im[k] - 1, 0);
                    gnode[k] = (ld(ip[0], ip[1], ip[2]) - ld(im[0], im[1], im[2])) * c.inv2h;
                    const double coef = (double)gbar[k] * (double)w * (double)c.inv2h;
                    atomicAdd(mu + node_index(f, ip[0], ip[1], ip[2]), coef);
                    atomicAdd(mu + node_index(f, im[0], im[1], im[2]), -coef);
                }
#pragma unroll
                for (int m = 0; m < DIM; ++m) {
                    float dwm = sg[m] * f.inv_h;
#pragma unroll
                    for (int q = 0; q < DIM; ++q)
                        if (q != m) dwm *= w1[q];
                    float s = 0.f;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) s = fmaf(gbar[k], gnode[k], s);
                    pb[m] = fmaf(dwm, s, pb[m]);
                }
            }
#pragma unroll
    for (int i = 0; i < DIM; ++i) pbar[i] = pb[i];
}

// One backward step of the cones (+ de_k += mu_in[cell_k] by the first threads).
template <int DIM>
__global__ void __launch_bounds__(256) adj_cone_kernel(FieldDesc f, ConeDesc c, const float *__restrict__ C,
                                                       uint32_t step, int n, const float *__restrict__ P,
                                                       const float *__restrict__ Dd,
                                                       const uint8_t *__restrict__ active, float *pbar,
                                                       float *dbar, double *mu_out, const double *__restrict__ mu_in,
                                                       const int32_t *__restrict__ src_cell, int n_src,
                                                       double *de_acc)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n_src) {
        const long long cell = src_cell[a];
        if (cell >= 0 && cell < (long long)f.nx * f.ny * f.nz) de_acc[a] += mu_in[cell];
    }
    if (a >= n || !active[a]) return;
    float p[DIM], d[DIM], pb[DIM], db[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        p[i] = P[(size_t)i * n + a];
        d[i] = Dd[(size_t)i * n + a];
        pb[i] = pbar[(size_t)i * n + a];
        db[i] = dbar[(size_t)i * n + a];
    }
    cone_adjoint<DIM>(f, c, C, (uint32_t)a, step, p, d, pb, db, mu_out);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        pbar[(size_t)i * n + a] = pb[i];
        dbar[(size_t)i * n + a] = db[i];
    }
}

// Loss and dL/dp^T = 2 (p^T - t)/n, dL/dd^T = 0.
__global__ void __launch_bounds__(256) adj_loss_kernel(int n, int dim, const float *__restrict__ P,
                                                       const float *__restrict__ T, float *pbar, float *dbar,
                                                       double *loss_acc)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (a < n) {
        for (int i = 0; i < dim; ++i) {
            const float e = P[(size_t)i * n + a] - T[(size_t)i * n + a];
            s += (double)e * (double)e;
            pbar[(size_t)i * n + a] = 2.0f * e / (float)n;
            dbar[(size_t)i * n + a] = 0.0f;
        }
    }
    block_add2(s, 0.0, loss_acc);
}

// Scale the accumulators into the caller's outputs.
__global__ void adj_finalize_kernel(FieldDesc f, int n_axons, const double *acc, int n_src, float *gD, float *gl,
                                    float *gsrc, float *loss, const double *S, float *gmap, size_t n_cells)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t == 0) {
        *gD = (float)((double)f.dt / ((double)f.h * f.h) * acc[0]);
        *gl = (float)(-(double)f.dt * acc[1]);
        *loss = (float)(acc[2 + n_src] / (n_axons > 0 ? n_axons : 1));
    }
    if (t < (size_t)n_src) gsrc[t] = (float)acc[2 + t];
    if (gmap)
        for (size_t c = t; c < n_cells; c += (size_t)gridDim.x * blockDim.x) gmap[c] = (float)((double)f.dt * S[c]);
}

struct AdjLayout {
    size_t ckpt_c, ckpt_p, seg_c, seg_p, mu, S, pbar, acc, total;
    int nseg;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

AdjLayout adj_layout(const cue_params &p, int n_src, int n_axons, int nsteps, int k)
{
    AdjLayout L{};
    const size_t cells = (size_t)p.nx * p.ny * (p.dim == 3 ? p.nz : 1);
    const size_t cone = (size_t)2 * p.dim * (n_axons > 0 ? n_axons : 1);    // pos + dir
    L.nseg = (nsteps + k - 1) / k;
    size_t off = 0;
    L.ckpt_c = off;
    off += align256(sizeof(float) * cells * L.nseg);
    L.ckpt_p = off;
    off += align256(sizeof(float) * cone * L.nseg);
    L.seg_c = off;
    off += align256(sizeof(float) * cells * (k + 1));
    L.seg_p = off;
    off += align256(sizeof(float) * cone * (k + 1));
    L.mu = off;                                   // FP64 adjoint field, two buffers
    off += align256(sizeof(double) * cells * 2);
    L.S = off;                                    // FP64 running sum of mu (rate-map gradient)
    off += align256(sizeof(double) * cells);
    L.pbar = off;
    off += align256(sizeof(float) * cone);
    L.acc = off;                                  // sD, sL, de[n_src], loss, spare
    off += align256(sizeof(double) * (4 + n_src));
    L.total = off;
    return L;
}

int blocks_for(size_t n, int per) { return (int)((n + per - 1) / per); }

}  // namespace

size_t adjoint_workspace_bytes(const cue_params &p, int n_src, int n_axons, int nsteps, int ckpt_every)
{
    if (nsteps <= 0 || ckpt_every <= 0) return 0;
    return adj_layout(p, n_src, n_axons, nsteps, ckpt_every).total;
}

int run_adjoint(Sim &s, const float *targets, int nsteps, int k, void *ws, size_t ws_bytes, float *gD, float *gl,
                float *gsrc, float *gmap, float *loss)
{
    const FieldDesc &f = s.fd;
    const size_t cells = (size_t)f.nx * f.ny * f.nz;
    const int n = s.n_axons, dim = f.dim;
    const size_t cone_n = (size_t)dim * n;                 // floats per pos (or dir) array
    AdjLayout L = adj_layout(s.params, s.n_src, n, nsteps, k);
    if (!ws || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255u)) return CUE_ERR_WORKSPACE;
    unsigned char *W = static_cast<unsigned char *>(ws);
    float *ckC = reinterpret_cast<float *>(W + L.ckpt_c);
    float *ckP = reinterpret_cast<float *>(W + L.ckpt_p);
    float *sgC = reinterpret_cast<float *>(W + L.seg_c);
    float *sgP = reinterpret_cast<float *>(W + L.seg_p);
    double *mu[2] = {reinterpret_cast<double *>(W + L.mu), reinterpret_cast<double *>(W + L.mu) + cells};
    double *S = gmap ? reinterpret_cast<double *>(W + L.S) : nullptr;
    float *pbar = reinterpret_cast<float *>(W + L.pbar), *dbar = pbar + cone_n;
    double *acc = reinterpret_cast<double *>(W + L.acc);     // sD, sL, de[n_src], loss
    cudaStream_t st = s.stream;
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    if (!ok(cudaMemsetAsync(mu[0], 0, sizeof(double) * cells * 2, st)) ||
        !ok(cudaMemsetAsync(acc, 0, sizeof(double) * (4 + s.n_src), st)) ||
        (S && !ok(cudaMemsetAsync(S, 0, sizeof(double) * cells, st))))
        return CUE_ERR_CUDA;
    const int64_t n0 = s.field_step;
    // ---- forward with checkpoints (any path: fused and plain agree bit for bit)
    for (int j = 0; j < L.nseg; ++j) {
        const int len = std::min(k, nsteps - j * k);
        if (!ok(cudaMemcpyAsync(ckC + cells * j, s.field[s.cur], sizeof(float) * cells, cudaMemcpyDeviceToDevice,
                                st)) ||
            !ok(cudaMemcpyAsync(ckP + 2 * cone_n * j, s.pos, sizeof(float) * cone_n, cudaMemcpyDeviceToDevice, st)) ||
            !ok(cudaMemcpyAsync(ckP + 2 * cone_n * j + cone_n, s.dir, sizeof(float) * cone_n,
                                cudaMemcpyDeviceToDevice, st)))
            return CUE_ERR_CUDA;
        int rc = run_coupled(s, len);
        if (rc != CUE_OK) return rc;
    }
    // ---- loss and its adjoint at the end
    if (n > 0) {
        adj_loss_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, dim, s.pos, targets, pbar, dbar, acc + 2 + s.n_src);
        s.launches++;
    }
    // ---- backwards through the segments
    int in = 0;
    for (int j = L.nseg - 1; j >= 0; --j) {
        const int len = std::min(k, nsteps - j * k);
        const int64_t nstart = n0 + (int64_t)j * k;
        if (!ok(cudaMemcpyAsync(sgC, ckC + cells * j, sizeof(float) * cells, cudaMemcpyDeviceToDevice, st)) ||
            !ok(cudaMemcpyAsync(sgP, ckP + 2 * cone_n * j, sizeof(float) * 2 * cone_n, cudaMemcpyDeviceToDevice, st)))
            return CUE_ERR_CUDA;
        for (int m = 0; m < len; ++m) {      // recompute, storing every step
            float *Pm = sgP + 2 * cone_n * m, *Pn = sgP + 2 * cone_n * (m + 1);
            if (!ok(launch_cone_step_io(s, sgC + cells * m, (uint32_t)(nstart + m), Pm, Pm + cone_n, Pn,
                                        Pn + cone_n)) ||
                !ok(launch_field_step(s, sgC + cells * m, sgC + cells * (m + 1))) ||
                !ok(launch_sources(s, sgC + cells * (m + 1))))
                return CUE_ERR_CUDA;
        }
        for (int m = len - 1; m >= 0; --m) {
            const float *Cm = sgC + cells * m, *Pm = sgP + 2 * cone_n * m;
            const int fb = std::min(blocks_for(cells, 256), 152 * 16);
            adj_field_kernel<<<fb, 256, 0, st>>>(f, mu[in], mu[in ^ 1], Cm, S, acc);
            s.launches++;
            const int cb = blocks_for((size_t)std::max(n, s.n_src), 256);
            if (cb > 0) {
                if (dim == 2)
                    adj_cone_kernel<2><<<cb, 256, 0, st>>>(f, s.cd, Cm, (uint32_t)(nstart + m), n, Pm, Pm + cone_n,
                                                           s.active, pbar, dbar, mu[in ^ 1], mu[in], s.src_cell,
                                                           s.n_src, acc + 2);
                else
                    adj_cone_kernel<3><<<cb, 256, 0, st>>>(f, s.cd, Cm, (uint32_t)(nstart + m), n, Pm, Pm + cone_n,
                                                           s.active, pbar, dbar, mu[in ^ 1], mu[in], s.src_cell,
                                                           s.n_src, acc + 2);
                s.launches++;
            }
            if (!ok(cudaGetLastError())) return CUE_ERR_CUDA;
            in ^= 1;
        }
    }
    adj_finalize_kernel<<<std::max(blocks_for((size_t)s.n_src, 256), std::min(blocks_for(cells, 256), 152 * 8)),
                          256, 0, st>>>(
        f, n, acc, s.n_src, gD, gl, gsrc, loss, S, gmap, cells);
    s.launches++;
    return ok(cudaGetLastError()) ? CUE_OK : CUE_ERR_CUDA;
}

}  // namespace cue
