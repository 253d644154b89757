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
// Memory: the forward keeps (C, p, d) every ckpt_every steps and runs its last
// segment as a stored trajectory; every other segment is recomputed from its
// checkpoint storing every step (one persistent launch on 2D grids with
// nx % 4 == 0, else a cone and a field launch per step).  With ckpt_every >=
// nsteps the whole run is stored once and nothing is recomputed.  Each segment
// is then walked backwards: one persistent cooperative launch per segment (adj_persist_kernel:
// field warps advance the adjoint field, cone warps scatter the cone adjoint,
// one bounded grid barrier per step), or, where that launch does not apply, a
// field launch and a cone launch per step.
//
// Precision: the adjoint field is double-float (two FP32 planes carried with
// error-free transformations, so GB300 runs it at FP32 rate); the cone reverse
// mode is FP64 at the FP32 forward values, with dL/d(p, d) kept in FP64; the
// per-thread partial sums of the dD and dlambda products are FP32, their block
// totals, the per-source sums and the segment totals of the rate-map sum
// FP64.
#include <algorithm>

#include "cue_barrier.cuh"
#include "cue_internal.h"

namespace cue {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

// Block sum of two per-thread FP32 partials: warps sum in FP32, the block
// total is formed in FP64 (GB300's FP64 rate is a small fraction of its FP32
// rate, so FP64 is kept to a few operations per block) and added to acc[0],
// acc[1].  PART: acc is this block's own pair of slots (a plain
// read-modify-write, no two blocks on one address, and the same sum order on
// every run); otherwise acc is shared and updated atomically.  Every thread of
// the block must call it.
template <bool PART>
__device__ __forceinline__ void block_add2(float a, float b, double *acc)
{
    __shared__ float sa[32], sb[32];
    const int t = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = t & 31, warp = t >> 5;
    a = warp_sumf(a);
    b = warp_sumf(b);
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x * blockDim.y + 31) / 32;
        double da = lane < nw ? (double)sa[lane] : 0.0;
        double db = lane < nw ? (double)sb[lane] : 0.0;
        da = warp_sum(da);
        db = warp_sum(db);
        if (lane == 0) {
            if (PART) {
                const size_t bid = blockIdx.x + (size_t)gridDim.x * blockIdx.y;
                acc[2 * bid] += da;
                acc[2 * bid + 1] += db;
            } else {
                atomicAdd(&acc[0], da);
                atomicAdd(&acc[1], db);
            }
        }
    }
}

// ---- double-float arithmetic (Dekker 1971; Knuth TAOCP vol. 2, 4.2.2):
// a value is an unevaluated sum hi + lo of two floats, and sums and products
// carry their rounding error forward with error-free transformations, all in
// FP32.  The explicit _rn intrinsics keep the compiler from contracting them.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return {s, e};
}

__device__ __forceinline__ DF quick_two_sum(float a, float b)      // |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// (a + b) with an absolute error of a few u^2 (|a| + |b|), u = 2^-24.
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    DF s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// a * c for a float c.
__device__ __forceinline__ DF df_mul(DF a, float c)
{
    const float p = __fmul_rn(a.hi, c);
    const float e = fmaf(a.lo, c, fmaf(a.hi, c, -p));
    return quick_two_sum(p, e);
}

__device__ __forceinline__ DF df_of(float hi, float lo) { return two_sum(hi, lo); }   // renormalise

// One backward field step on an nx % 4 == 0 2D grid, laid out like the
// forward's float4 kernel (32 lanes x 4 nodes in x, 8 warps of `rows` rows):
//   mu_out = A mu_in (A is the forward stencil: the no-flux operator is
//   symmetric),  acc[0] += <lap(mu_in), C>,  acc[1] += <mu_in, C>,
//   Sseg += mu_in (the rate-map sum of this segment).
// mu is double-float: a buffer holds the high plane, then the low plane.
// Cones near the diffusion front, where |grad C| is tiny, scatter large
// contributions of opposite sign into neighbouring nodes that the stencil
// then cancels; a single float would keep only their rounding errors.
__device__ __forceinline__ DF df_update(DF m, DF l, DF r, DF u, DF d, float alpha, float beta, float *lap)
{
    const DF sum = df_add(df_add(l, r), df_add(u, d));
    const DF lp = df_add(sum, df_mul(m, -4.0f));
    *lap = lp.hi + lp.lo;
    return df_add(df_mul(m, beta), df_mul(sum, alpha));
}

// The segment's rate-map sum of four nodes, Sseg += mu, as a double-float (high
// and low planes): the adjoint at a source or in a cone's orbit swings between
// large values of either sign from step to step, and their sum is a small
// remainder that a single float would hold only to its rounding.
__device__ __forceinline__ void seg_sum_add(float4 *hi, float4 *lo, const DF &m0, const DF &m1, const DF &m2,
                                            const DF &m3)
{
    const float4 h = *hi, l = *lo;
    const DF a0 = df_add(df_of(h.x, l.x), m0), a1 = df_add(df_of(h.y, l.y), m1);
    const DF a2 = df_add(df_of(h.z, l.z), m2), a3 = df_add(df_of(h.w, l.w), m3);
    *hi = make_float4(a0.hi, a1.hi, a2.hi, a3.hi);
    *lo = make_float4(a0.lo, a1.lo, a2.lo, a3.lo);
}

__global__ void __launch_bounds__(256) adj_field2d_vec4(FieldDesc f, const float *__restrict__ mu_in,
                                                        float *__restrict__ mu_out, const float *__restrict__ C,
                                                        float *Sseg, double *acc, int rows)
{
    const int lane = threadIdx.x;
    const int nx4 = f.nx >> 2;
    const size_t cells = (size_t)f.nx * f.ny;
    const int x4 = blockIdx.x * 32 + lane;
    const int y0 = (blockIdx.y * blockDim.y + threadIdx.y) * rows;
    const bool act = x4 < nx4 && y0 < f.ny;
    const int y1 = min(y0 + rows, f.ny);
    const int x = x4 * 4;
    const bool has_l = x > 0, has_r = x + 4 < f.nx;
    const float4 *hi4 = reinterpret_cast<const float4 *>(mu_in);
    const float4 *lo4 = reinterpret_cast<const float4 *>(mu_in + cells);
    const float4 *c4 = reinterpret_cast<const float4 *>(C);
    float4 *ohi4 = reinterpret_cast<float4 *>(mu_out);
    float4 *olo4 = reinterpret_cast<float4 *>(mu_out + cells);
    float4 *s4 = reinterpret_cast<float4 *>(Sseg);
    float4 *s4lo = reinterpret_cast<float4 *>(Sseg + cells);
    float tD = 0.f, tL = 0.f;
    if (y0 < f.ny) {                               // warp-uniform
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        auto row = [&](int y, float4 &h, float4 &l) {
            h = __ldg(hi4 + (size_t)y * nx4 + x4);
            l = __ldg(lo4 + (size_t)y * nx4 + x4);
        };
        float4 ch = z4, cl = z4, uh, ul;
        if (act) row(y0, ch, cl);
        uh = ch;
        ul = cl;
        if (act && y0 > 0) row(y0 - 1, uh, ul);
        for (int y = y0; y < y1; ++y) {
            float4 dh = ch, dl = cl;
            if (act && y + 1 < f.ny) row(y + 1, dh, dl);
            float lh = __shfl_up_sync(kFull, ch.w, 1), ll = __shfl_up_sync(kFull, cl.w, 1);
            float rh = __shfl_down_sync(kFull, ch.x, 1), rl = __shfl_down_sync(kFull, cl.x, 1);
            if (lane == 0) {
                const bool e = act && has_l;
                lh = e ? __ldg(mu_in + (size_t)y * f.nx + x - 1) : ch.x;
                ll = e ? __ldg(mu_in + cells + (size_t)y * f.nx + x - 1) : cl.x;
            }
            if (lane == 31) {
                const bool e = act && has_r;
                rh = e ? __ldg(mu_in + (size_t)y * f.nx + x + 4) : ch.w;
                rl = e ? __ldg(mu_in + cells + (size_t)y * f.nx + x + 4) : cl.w;
            }
            if (!has_l) {
                lh = ch.x;
                ll = cl.x;
            }
            if (!has_r) {
                rh = ch.w;
                rl = cl.w;
            }
            if (act) {
                const size_t at = (size_t)y * nx4 + x4;
                const float4 c = __ldg(c4 + at);
                const DF m0 = df_of(ch.x, cl.x), m1 = df_of(ch.y, cl.y), m2 = df_of(ch.z, cl.z),
                         m3 = df_of(ch.w, cl.w);
                float L0, L1, L2, L3;
                const DF o0 = df_update(m0, df_of(lh, ll), m1, df_of(uh.x, ul.x), df_of(dh.x, dl.x), f.alpha,
                                        f.beta, &L0);
                const DF o1 = df_update(m1, m0, m2, df_of(uh.y, ul.y), df_of(dh.y, dl.y), f.alpha, f.beta, &L1);
                const DF o2 = df_update(m2, m1, m3, df_of(uh.z, ul.z), df_of(dh.z, dl.z), f.alpha, f.beta, &L2);
                const DF o3 = df_update(m3, m2, df_of(rh, rl), df_of(uh.w, ul.w), df_of(dh.w, dl.w), f.alpha,
                                        f.beta, &L3);
                const float v0 = m0.hi + m0.lo, v1 = m1.hi + m1.lo, v2 = m2.hi + m2.lo, v3 = m3.hi + m3.lo;
                tD = fmaf(L0, c.x, fmaf(L1, c.y, fmaf(L2, c.z, fmaf(L3, c.w, tD))));
                tL = fmaf(v0, c.x, fmaf(v1, c.y, fmaf(v2, c.z, fmaf(v3, c.w, tL))));
                if (Sseg) seg_sum_add(s4 + at, s4lo + at, m0, m1, m2, m3);
                ohi4[at] = make_float4(o0.hi, o1.hi, o2.hi, o3.hi);
                olo4[at] = make_float4(o0.lo, o1.lo, o2.lo, o3.lo);
            }
            uh = ch;
            ul = cl;
            ch = dh;
            cl = dl;
        }
    }
    block_add2<true>(tD, tL, acc);
}

// The same for any grid (2D or 3D, any nx), one node per thread iteration.
__global__ void __launch_bounds__(256) adj_field_scalar(FieldDesc f, const float *__restrict__ mu_in,
                                                        float *__restrict__ mu_out, const float *__restrict__ C,
                                                        float *Sseg, double *acc)
{
    const size_t n = (size_t)f.nx * f.ny * f.nz;
    const size_t sy = f.nx, sz = (size_t)f.nx * f.ny;
    float tD = 0.f, tL = 0.f;
    auto ld = [&](size_t c) { return df_of(mu_in[c], mu_in[n + c]); };
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % f.nx);
        const int j = (int)((c / f.nx) % f.ny);
        const int k = (int)(c / sz);
        const DF m = ld(c);
        const DF xm = i > 0 ? ld(c - 1) : m;
        const DF xp = i < f.nx - 1 ? ld(c + 1) : m;
        const DF ym = j > 0 ? ld(c - sy) : m;
        const DF yp = j < f.ny - 1 ? ld(c + sy) : m;
        DF sum = df_add(df_add(xm, xp), df_add(ym, yp));
        float nn = -4.0f;
        if (f.dim == 3) {
            const DF zm = k > 0 ? ld(c - sz) : m;
            const DF zp = k < f.nz - 1 ? ld(c + sz) : m;
            sum = df_add(sum, df_add(zm, zp));
            nn = -6.0f;
        }
        const DF lp = df_add(sum, df_mul(m, nn));
        const DF o = df_add(df_mul(m, f.beta), df_mul(sum, f.alpha));
        const float v = m.hi + m.lo;
        const float cc = C[c];
        tD = fmaf(lp.hi + lp.lo, cc, tD);
        tL = fmaf(v, cc, tL);
        if (Sseg) {
            const DF sv = df_add(df_of(Sseg[c], Sseg[n + c]), m);
            Sseg[c] = sv.hi;
            Sseg[n + c] = sv.lo;
        }
        mu_out[c] = o.hi;
        mu_out[n + c] = o.lo;
    }
    block_add2<true>(tD, tL, acc);
}

// End of a segment: S += Sseg in FP64 (Sseg double-float: high plane, then
// low plane), Sseg = 0.
__global__ void __launch_bounds__(256) adj_fold_kernel(size_t n, float *Sseg, double *S)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
        S[c] += (double)Sseg[c] + (double)Sseg[n + c];
        Sseg[c] = 0.0f;
        Sseg[n + c] = 0.0f;
    }
}

// Node (i,j,k) as a linear index.
__device__ __forceinline__ size_t node_index(const FieldDesc &f, int i, int j, int k)
{
    return (size_t)i + (size_t)f.nx * ((size_t)j + (size_t)f.ny * k);
}

// Backward through one clamp-mode 2D cone step.  p, d: state at step n;
// pbar, dbar: in dL/d(p,d)^{n+1}, out dL/d(p,d)^n; the field part is
// scattered into mu.  The 12-node patch gathered for the forward recomputation
// also gives the corner node gradients (position derivative), and the field
// adjoint is summed per patch node in registers, then scattered with 12
// independent double-float atomics (instead of reloading the nodes and
// scattering 16 pairs corner by corner).  pbar and dbar are FP64.  Patch slots are gather2's:
//   0..3 (xm, x0, x1, xp) at y0;  4..7 the same at y1;  8, 9 (x0, x1) at ym;
//   10, 11 (x0, x1) at yp.
// 1/sqrt(x) in FP64 for x in the normal float range: a float seed and two
// Newton steps y <- y (3 - x y^2) / 2 (relative error about 1e-14), far fewer
// FP64 instructions than an IEEE square root and division.
__device__ __forceinline__ double rsqrt_d(double x)
{
    double y = (double)rsqrtf((float)x);
    y = y * (1.5 - 0.5 * x * y * y);
    return y * (1.5 - 0.5 * x * y * y);
}

// Double-float accumulation of an FP64 value c into (hi, lo): c rounded to
// FP32 goes to the high plane; its rounding error plus the exact rounding
// error of that add (recovered from the returned old value, as the atomic
// rounds to nearest) goes to the low plane.  Whatever the order of the
// atomics, hi + sum(lo) stays the exact sum up to the low plane's rounding.
__device__ __forceinline__ void atomic_add_df64(float *hi, float *lo, double c)
{
    const float ch = (float)c;
    const float old = atomicAdd(hi, ch);
    const float r = two_sum(old, ch).lo + (float)(c - (double)ch);
    if (r != 0.0f) atomicAdd(lo, r);
}

// Backward through one clamp-mode 3D cone step, the reverse mode in FP64 at
// the FP32 state it is given (the decisions -- gradient threshold, blend
// threshold, clamp -- and the noise are the FP32 forward's; inv_hd = 1/h in
// FP64).  pbar, dbar: FP64, in dL/d(p,
// d)^{n+1}, out dL/d(p, d)^n; the field part is scattered into mu.
__device__ __forceinline__ void cone_adjoint3(const FieldDesc &f, const ConeDesc &c, double inv_hd,
                                              const float *__restrict__ C, uint32_t axon, uint32_t step,
                                              const float *p, const float *d, double *pbar, double *dbar, float *mu)
{
    constexpr int DIM = 3;
    const size_t sy = f.nx, sz = (size_t)f.nx * f.ny;
    float *mu_lo = mu + sz * f.nz;
    auto ld = [&](int i, int j, int k) { return __ldg(C + (size_t)i + sy * j + sz * k); };
    // the forward step in FP32, for its decisions
    float g[DIM], xi[DIM];
    sample_gradient<DIM>(f, c, p, ld, g);
    cone_noise<DIM>(c.key0, c.key1, axon, step, xi);
    float gn2 = 0.f;
#pragma unroll
    for (int i = 0; i < DIM; ++i) gn2 = fmaf(g[i], g[i], gn2);
    const bool has_g = gn2 > c.eps2;
    const float ginv = has_g ? rsqrtf(gn2) : 0.0f;
    float vf[DIM], vn2 = 0.f;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        vf[i] = c.w_prev * d[i] + c.w_grad * (g[i] * ginv) + c.w_noise * xi[i];
        vn2 = fmaf(vf[i], vf[i], vn2);
    }
    const bool has_v = vn2 > 1e-30f;
    const float vinv = has_v ? rsqrtf(vn2) : 0.0f;
    const float hi[3] = {c.hi0, c.hi1, c.hi2};
    bool clamped[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        const float q = fmaf(c.step_len, has_v ? vf[i] * vinv : d[i], p[i]);
        clamped[i] = q < 0.0f || q > hi[i];
    }
    // the sample in FP64: cell, fractions, corner node gradients, weights
    int lo[3] = {0, 0, 0};
    float frf[3] = {0.f, 0.f, 0.f};
    cell_of<DIM>(f, p, lo, frf);
    const int ext[3] = {f.nx, f.ny, f.nz};
    const double i2h = (double)c.inv2h;
    double fr[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) fr[i] = (double)p[i] * inv_hd - (double)lo[i];
    double G[8][DIM], W[8];
    double gd[DIM] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int cidx = 0; cidx < 8; ++cidx) {
        const int a = cidx & 1, b = (cidx >> 1) & 1, e = cidx >> 2;
        const int idx[3] = {lo[0] + a, lo[1] + b, lo[2] + e};
        W[cidx] = (a ? fr[0] : 1.0 - fr[0]) * (b ? fr[1] : 1.0 - fr[1]) * (e ? fr[2] : 1.0 - fr[2]);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            int ip[3] = {idx[0], idx[1], idx[2]}, im[3] = {idx[0], idx[1], idx[2]};
            ip[k] = min(ip[k] + 1, ext[k] - 1);
            im[k] = max(im[k] - 1, 0);
            G[cidx][k] = ((double)ld(ip[0], ip[1], ip[2]) - (double)ld(im[0], im[1], im[2])) * i2h;
            gd[k] += W[cidx] * G[cidx][k];
        }
    }
    double ghat[DIM] = {0.0, 0.0, 0.0}, ginvd = 0.0;
    if (has_g) {
        ginvd = rsqrt_d(gd[0] * gd[0] + gd[1] * gd[1] + gd[2] * gd[2]);
#pragma unroll
        for (int i = 0; i < DIM; ++i) ghat[i] = gd[i] * ginvd;
    }
    double vd[DIM], dn[DIM], vinvd = 0.0;
#pragma unroll
    for (int i = 0; i < DIM; ++i)
        vd[i] = (double)c.w_prev * (double)d[i] + (double)c.w_grad * ghat[i] + (double)c.w_noise * (double)xi[i];
    if (has_v) vinvd = rsqrt_d(vd[0] * vd[0] + vd[1] * vd[1] + vd[2] * vd[2]);
#pragma unroll
    for (int i = 0; i < DIM; ++i) dn[i] = has_v ? vd[i] * vinvd : (double)d[i];
    double qbar[DIM], dnbar[DIM], vbar[DIM], gbar[DIM] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        qbar[i] = clamped[i] ? 0.0 : pbar[i];
        dnbar[i] = (double)c.step_len * qbar[i] + dbar[i];
    }
    if (has_v) {
        const double dot = dn[0] * dnbar[0] + dn[1] * dnbar[1] + dn[2] * dnbar[2];
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            vbar[i] = (dnbar[i] - dn[i] * dot) * vinvd;
            dbar[i] = (double)c.w_prev * vbar[i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            vbar[i] = 0.0;
            dbar[i] = dnbar[i];
        }
    }
    if (has_g) {
        const double wg = (double)c.w_grad;
        const double dot = ghat[0] * (wg * vbar[0]) + ghat[1] * (wg * vbar[1]) + ghat[2] * (wg * vbar[2]);
#pragma unroll
        for (int i = 0; i < DIM; ++i) gbar[i] = (wg * vbar[i] - ghat[i] * dot) * ginvd;
    }
    // back through the sample: position (weight derivatives) and field (node differences)
    double pb[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) pb[i] = qbar[i];
    const double ih = inv_hd;
#pragma unroll
    for (int cidx = 0; cidx < 8; ++cidx) {
        const int a = cidx & 1, b = (cidx >> 1) & 1, e = cidx >> 2;
        const double w1[3] = {a ? fr[0] : 1.0 - fr[0], b ? fr[1] : 1.0 - fr[1], e ? fr[2] : 1.0 - fr[2]};
        const double sg[3] = {a ? 1.0 : -1.0, b ? 1.0 : -1.0, e ? 1.0 : -1.0};
        const double sdot = gbar[0] * G[cidx][0] + gbar[1] * G[cidx][1] + gbar[2] * G[cidx][2];
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
            double dwm = sg[m] * ih;
#pragma unroll
            for (int q = 0; q < DIM; ++q)
                if (q != m) dwm *= w1[q];
            pb[m] += dwm * sdot;
        }
        if (!has_g) continue;
        const int idx[3] = {lo[0] + a, lo[1] + b, lo[2] + e};
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            int ip[3] = {idx[0], idx[1], idx[2]}, im[3] = {idx[0], idx[1], idx[2]};
            ip[k] = min(ip[k] + 1, ext[k] - 1);
            im[k] = max(im[k] - 1, 0);
            const double coef = gbar[k] * W[cidx] * i2h;
            const size_t jp = node_index(f, ip[0], ip[1], ip[2]), jm = node_index(f, im[0], im[1], im[2]);
            atomic_add_df64(mu + jp, mu_lo + jp, coef);
            atomic_add_df64(mu + jm, mu_lo + jm, -coef);
        }
    }
#pragma unroll
    for (int i = 0; i < DIM; ++i) pbar[i] = pb[i];
}

__device__ __forceinline__ void cone_adjoint2(const FieldDesc &f, const ConeDesc &c, double inv_hd,
                                              const float *__restrict__ C, uint32_t axon, uint32_t step,
                                              const float *p, const float *d, double *pbar, double *dbar, float *mu)
{
    const size_t sy = f.nx;
    auto ld = [&](int i, int j, int) { return __ldg(C + (size_t)i + sy * j); };
    // the forward step in FP32, for its decisions (gradient threshold, blend
    // threshold, clamp) and the values it stepped from
    float xi[2];
    cone_noise<2>(c.key0, c.key1, axon, step, xi);
    int lo[3] = {0, 0, 0};
    float fr[3] = {0.f, 0.f, 0.f};
    cell_of<2>(f, p, lo, fr);
    float v[kPatch2];
    gather2(f, lo, ld, v);
    float g[2];
    grad2(c, v, fr, g);                                   // the forward's gradient, bit for bit
    const float gn2 = fmaf(g[1], g[1], g[0] * g[0]);
    const bool has_g = gn2 > c.eps2;
    const float ginv = has_g ? rsqrtf(gn2) : 0.0f;
    float vv[2], vn2 = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        vv[i] = c.w_prev * d[i] + c.w_grad * (g[i] * ginv) + c.w_noise * xi[i];
        vn2 = fmaf(vv[i], vv[i], vn2);
    }
    const bool has_v = vn2 > 1e-30f;
    const float vinv = has_v ? rsqrtf(vn2) : 0.0f;
    bool clamped[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float dnf = has_v ? vv[i] * vinv : d[i];
        const float q = fmaf(c.step_len, dnf, p[i]);
        clamped[i] = q < 0.0f || q > (i ? c.hi1 : c.hi0);
    }
    // the reverse mode in FP64 at that state: the adjoint of the endpoint loss
    // cancels heavily between cones and steps, and near a cue maximum or a
    // source the sampled gradient is a small difference of larger node values,
    // so the linearisation point -- sample and normalised gradient -- is formed
    // in FP64 from the FP32 node values and position (inv_hd = 1/h in FP64);
    // the per-cone work is small next to the field's
    const double i2h = (double)c.inv2h;
    const double frx = (double)p[0] * inv_hd - (double)lo[0], fry = (double)p[1] * inv_hd - (double)lo[1];
    const double wx0 = 1.0 - frx, wx1 = frx, wy0 = 1.0 - fry, wy1 = fry;
    const double w00 = wx0 * wy0, w10 = wx1 * wy0, w01 = wx0 * wy1, w11 = wx1 * wy1;
    const double gx00 = ((double)v[2] - v[0]) * i2h, gx10 = ((double)v[3] - v[1]) * i2h;
    const double gx01 = ((double)v[6] - v[4]) * i2h, gx11 = ((double)v[7] - v[5]) * i2h;
    const double gy00 = ((double)v[5] - v[8]) * i2h, gy10 = ((double)v[6] - v[9]) * i2h;
    const double gy01 = ((double)v[10] - v[1]) * i2h, gy11 = ((double)v[11] - v[2]) * i2h;
    const double gd[2] = {w00 * gx00 + w10 * gx10 + w01 * gx01 + w11 * gx11,
                          w00 * gy00 + w10 * gy10 + w01 * gy01 + w11 * gy11};
    double ghat[2] = {0.0, 0.0}, ginvd = 0.0;
    if (has_g) {
        ginvd = rsqrt_d(gd[0] * gd[0] + gd[1] * gd[1]);
        ghat[0] = gd[0] * ginvd;
        ghat[1] = gd[1] * ginvd;
    }
    double vd[2], dn[2], vinvd = 0.0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
        vd[i] = (double)c.w_prev * (double)d[i] + (double)c.w_grad * ghat[i] + (double)c.w_noise * (double)xi[i];
    if (has_v) vinvd = rsqrt_d(vd[0] * vd[0] + vd[1] * vd[1]);
#pragma unroll
    for (int i = 0; i < 2; ++i) dn[i] = has_v ? vd[i] * vinvd : (double)d[i];
    double qbar[2], dnbar[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        qbar[i] = clamped[i] ? 0.0 : pbar[i];
        dnbar[i] = (double)c.step_len * qbar[i] + dbar[i];
    }
    double vbar[2];
    if (has_v) {
        const double dot = dn[0] * dnbar[0] + dn[1] * dnbar[1];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            vbar[i] = (dnbar[i] - dn[i] * dot) * vinvd;
            dbar[i] = (double)c.w_prev * vbar[i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            vbar[i] = 0.0;
            dbar[i] = dnbar[i];
        }
    }
    double gbar[2] = {0.0, 0.0};
    if (has_g) {
        const double wg = (double)c.w_grad;
        const double dot = ghat[0] * (wg * vbar[0]) + ghat[1] * (wg * vbar[1]);
#pragma unroll
        for (int i = 0; i < 2; ++i) gbar[i] = (wg * vbar[i] - ghat[i] * dot) * ginvd;
    }
    // position: g(p) = sum_c w_c(p) G_c (corner (a, b) = node (x_a, y_b)), dw/dp
    // from the bilinear weights
    const double s00 = gbar[0] * gx00 + gbar[1] * gy00, s10 = gbar[0] * gx10 + gbar[1] * gy10;
    const double s01 = gbar[0] * gx01 + gbar[1] * gy01, s11 = gbar[0] * gx11 + gbar[1] * gy11;
    const double ih = inv_hd;
    pbar[0] = ih * (wy0 * (s10 - s00) + wy1 * (s11 - s01)) + qbar[0];
    pbar[1] = ih * (wx0 * (s01 - s00) + wx1 * (s11 - s10)) + qbar[1];
    if (!has_g) return;
    // field: coefficient of each patch node in gbar . g
    const double ax = gbar[0] * i2h, ay = gbar[1] * i2h;
    const double cx00 = ax * w00, cx10 = ax * w10, cx01 = ax * w01, cx11 = ax * w11;
    const double cy00 = ay * w00, cy10 = ay * w10, cy01 = ay * w01, cy11 = ay * w11;
    const double sc[kPatch2] = {-cx00,        -cx10 - cy01, cx00 - cy11, cx10,
                                -cx01,        cy00 - cx11,  cy10 + cx01, cx11,
                                -cy00,        -cy10,        cy01,        cy11};
    const int xm = max(lo[0] - 1, 0), x0 = lo[0], x1 = lo[0] + 1, xp = min(lo[0] + 2, f.nx - 1);
    const int ym = max(lo[1] - 1, 0), y0 = lo[1], y1 = lo[1] + 1, yp = min(lo[1] + 2, f.ny - 1);
    const int xs[kPatch2] = {xm, x0, x1, xp, xm, x0, x1, xp, x0, x1, x0, x1};
    const int ys[kPatch2] = {y0, y0, y0, y0, y1, y1, y1, y1, ym, ym, yp, yp};
    float *mu_lo = mu + sy * f.ny;
    // double-float accumulation of an FP64 coefficient c: add ch = fl(c) to
    // the high plane, then the rounding error of that add (from the returned
    // old value) plus c - ch to the low plane; the twelve high-plane adds are
    // issued before the first returned value is used, so they are in flight
    // together
    float ch[kPatch2], old[kPatch2];
#pragma unroll
    for (int k = 0; k < kPatch2; ++k) {
        ch[k] = (float)sc[k];
        old[k] = atomicAdd(mu + (size_t)xs[k] + sy * ys[k], ch[k]);
    }
#pragma unroll
    for (int k = 0; k < kPatch2; ++k) {
        const float cl = (float)(sc[k] - (double)ch[k]);
        const float r = two_sum(old[k], ch[k]).lo + cl;
        if (r != 0.0f) atomicAdd(mu_lo + (size_t)xs[k] + sy * ys[k], r);
    }
}

// ---------------------------------------------------------------- persistent backward
// The cone adjoint never reads the adjoint field: going back through step m,
//   mu^m = A mu^{m+1} + X^m,   X^m = the cones' scatter at step m.
// With Y^m = A mu^{m+1}, one phase per step computes Y^m from
// mu^{m+1} = Y^{m+1} + X^{m+1} (field tiles) while the cone chunks scatter X^m,
// then the blocks meet at the grid barrier.  Y ping-pongs; X rotates over
// three buffers: a phase reads X^{m+1}, writes X^m and zeroes X^{m+2}, which
// the previous phase read and the next one writes.  All are double-float
// (hi plane, lo plane).  A segment's backward steps are one cooperative launch.
struct AdjP {
    FieldDesc f;
    ConeDesc c;
    double inv_h64;               // 1/h in FP64 (the cone reverse mode)
    int n;                        // cones
    int n_src;
    const int32_t *src_cell;
    const uint8_t *active;
    double *pbar, *dbar;          // dL/d(p, d), FP64
    const float *segC;            // [k + 1][cells]
    const float *segP;            // [k + 1][pos, dir][2][n]
    size_t cells, cone_n;
    float *Y[2];
    float *X[3];
    float *Sseg;                  // nullable
    double *part;                 // per-block (dD, dlambda) slots
    double *de;                   // per-source sums
    int ntx, n_chunks;
    int n_cone_warps, n_row_warps;
};

__device__ __forceinline__ DF mu_load(const float *Y, const float *X, size_t cells, size_t i)
{
    return df_add(df_of(__ldcg(Y + i), __ldcg(Y + cells + i)), df_of(__ldcg(X + i), __ldcg(X + cells + i)));
}

// One row of mu = Y + X as it is read (hi and lo planes of Y and X; lanes 0
// and 31 also the column beyond their end of the row).
struct AdjRow {
    float4 yh, yl, xh, xl;
    float e[4];                  // lane 0: column x - 1, lane 31: column x + 4 (yh, yl, xh, xl)
};

__device__ __forceinline__ void adj_row_load(const AdjP &A, const float *Yin, const float *Xin, int y, int x4,
                                             bool xin, bool has_l, bool has_r, AdjRow &R)
{
    const int lane = threadIdx.x & 31;
    const size_t cells = A.cells;
    const int nx4 = A.f.nx >> 2;
    const size_t at = (size_t)y * nx4 + x4;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    R.yh = xin ? __ldcg(reinterpret_cast<const float4 *>(Yin) + at) : z4;
    R.yl = xin ? __ldcg(reinterpret_cast<const float4 *>(Yin + cells) + at) : z4;
    R.xh = xin ? __ldcg(reinterpret_cast<const float4 *>(Xin) + at) : z4;
    R.xl = xin ? __ldcg(reinterpret_cast<const float4 *>(Xin + cells) + at) : z4;
    R.e[0] = R.e[1] = R.e[2] = R.e[3] = 0.f;
    const bool edge = (lane == 0 && has_l) || (lane == 31 && has_r);
    if (xin && edge) {
        const size_t i = (size_t)y * A.f.nx + 4 * x4 + (lane == 0 ? -1 : 4);
        R.e[0] = __ldcg(Yin + i);
        R.e[1] = __ldcg(Yin + cells + i);
        R.e[2] = __ldcg(Xin + i);
        R.e[3] = __ldcg(Xin + cells + i);
    }
}

// mu of a loaded row and the neighbours of its first and last node (Y is
// stored normalised by the tiles, X's planes take atomics and are
// renormalised).  Every lane of the warp calls it (shuffles).
__device__ __forceinline__ void adj_row_mu(const AdjRow &R, bool has_l, bool has_r, DF *m, DF &l, DF &r)
{
    const int lane = threadIdx.x & 31;
    m[0] = df_add(DF{R.yh.x, R.yl.x}, df_of(R.xh.x, R.xl.x));
    m[1] = df_add(DF{R.yh.y, R.yl.y}, df_of(R.xh.y, R.xl.y));
    m[2] = df_add(DF{R.yh.z, R.yl.z}, df_of(R.xh.z, R.xl.z));
    m[3] = df_add(DF{R.yh.w, R.yl.w}, df_of(R.xh.w, R.xl.w));
    l.hi = __shfl_up_sync(kFull, m[3].hi, 1);
    l.lo = __shfl_up_sync(kFull, m[3].lo, 1);
    r.hi = __shfl_down_sync(kFull, m[0].hi, 1);
    r.lo = __shfl_down_sync(kFull, m[0].lo, 1);
    const DF e = df_add(DF{R.e[0], R.e[1]}, df_of(R.e[2], R.e[3]));
    if (lane == 0) l = e;
    if (lane == 31) r = e;
    if (!has_l) l = m[0];
    if (!has_r) r = m[3];
}

// Backward update of one node: Y = beta mu + alpha (sum of the four
// neighbours), *lap = (sum - 4 mu) rounded to one float (the high part of its
// double-float sum plus the low part, which is what adding the two parts of a
// renormalised sum gives).
__device__ __forceinline__ DF df_update2(DF m, DF l, DF r, DF u, DF d, float alpha, float beta, float *lap)
{
    const DF sum = df_add(df_add(l, r), df_add(u, d));
    const DF s = two_sum(sum.hi, -4.0f * m.hi);
    *lap = __fadd_rn(s.hi, __fadd_rn(s.lo, __fadd_rn(sum.lo, -4.0f * m.lo)));
    return df_add(df_mul(m, beta), df_mul(sum, alpha));
}

// Rows ybeg .. yend - 1 of column strip tx (128 columns: 32 lanes x 4) of one
// backward step, by one warp streaming down y, so every row's mu is formed
// once (yend - ybeg + 2 rows read for yend - ybeg rows written).
__device__ __forceinline__ void adj_rows(const AdjP &A, const float *Yin, const float *Xin, float *Yout, float *Xz,
                                         const float *Cm, int tx, int ybeg, int yend, float &tD, float &tL)
{
    const FieldDesc &f = A.f;
    const int lane = threadIdx.x & 31;
    const int nx4 = f.nx >> 2;
    const int x4 = tx * 32 + lane;
    if (ybeg >= yend) return;                              // warp-uniform
    const bool xin = x4 < nx4;
    const int x = x4 * 4;
    const bool has_l = x > 0, has_r = x + 4 < f.nx;
    const size_t cells = A.cells;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    AdjRow ru, rc, rd;                                     // rows y - 1, y, y + 1 (walls repeat y)
    adj_row_load(A, Yin, Xin, ybeg > 0 ? ybeg - 1 : ybeg, x4, xin, has_l, has_r, ru);
    adj_row_load(A, Yin, Xin, ybeg, x4, xin, has_l, has_r, rc);
    adj_row_load(A, Yin, Xin, ybeg + 1 < f.ny ? ybeg + 1 : ybeg, x4, xin, has_l, has_r, rd);
    DF up[4], cu[4], dn[4], l, r, tl, tr;
    adj_row_mu(ru, has_l, has_r, up, tl, tr);
    adj_row_mu(rc, has_l, has_r, cu, l, r);
    for (int y = ybeg; y < yend; ++y) {
        // the row below the next one is on its way while this one is computed
        const int yn = y + 2 < f.ny ? y + 2 : f.ny - 1;
        AdjRow rn;
        if (y + 1 < yend) adj_row_load(A, Yin, Xin, yn, x4, xin, has_l, has_r, rn);
        adj_row_mu(rd, has_l, has_r, dn, tl, tr);
        const size_t at = (size_t)y * nx4 + x4;
        if (xin) {
            const float4 c = __ldg(reinterpret_cast<const float4 *>(Cm) + at);
            float4 *s4 = A.Sseg ? reinterpret_cast<float4 *>(A.Sseg) + at : nullptr;
            float L0, L1, L2, L3;
            const DF o0 = df_update2(cu[0], l, cu[1], up[0], dn[0], f.alpha, f.beta, &L0);
            const DF o1 = df_update2(cu[1], cu[0], cu[2], up[1], dn[1], f.alpha, f.beta, &L1);
            const DF o2 = df_update2(cu[2], cu[1], cu[3], up[2], dn[2], f.alpha, f.beta, &L2);
            const DF o3 = df_update2(cu[3], cu[2], r, up[3], dn[3], f.alpha, f.beta, &L3);
            const float v0 = cu[0].hi + cu[0].lo, v1 = cu[1].hi + cu[1].lo, v2 = cu[2].hi + cu[2].lo,
                        v3 = cu[3].hi + cu[3].lo;
            tD = fmaf(L0, c.x, fmaf(L1, c.y, fmaf(L2, c.z, fmaf(L3, c.w, tD))));
            tL = fmaf(v0, c.x, fmaf(v1, c.y, fmaf(v2, c.z, fmaf(v3, c.w, tL))));
            if (s4) seg_sum_add(s4, reinterpret_cast<float4 *>(A.Sseg + cells) + at, cu[0], cu[1], cu[2], cu[3]);
            reinterpret_cast<float4 *>(Yout)[at] = make_float4(o0.hi, o1.hi, o2.hi, o3.hi);
            reinterpret_cast<float4 *>(Yout + cells)[at] = make_float4(o0.lo, o1.lo, o2.lo, o3.lo);
            reinterpret_cast<float4 *>(Xz)[at] = z4;
            reinterpret_cast<float4 *>(Xz + cells)[at] = z4;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            up[i] = cu[i];
            cu[i] = dn[i];
        }
        l = tl;
        r = tr;
        if (y + 1 < yend) rd = rn;
    }
}

__global__ void __launch_bounds__(256, 2) adj_persist_kernel(AdjP A, int len, uint32_t g0, PBar *bar,
                                                             unsigned expected, long long limit, unsigned *status)
{
    // each thread's dD and dlambda products, summed over the segment's steps in
    // compensated FP32 (two_sum: hi + lo), reduced over the block once at the end
    DF sD{0.f, 0.f}, sL{0.f, 0.f};
    for (int m = len - 1; m >= 0; --m) {
        const uint32_t g = g0 + (uint32_t)m;              // global step index
        const float *Yin = A.Y[(g + 1) & 1];
        float *Yout = A.Y[g & 1];
        const float *Xin = A.X[(g + 1) % 3];
        float *Xout = A.X[g % 3];
        float *Xz = A.X[(g + 2) % 3];
        const float *Cm = A.segC + A.cells * m;
        const float *Pm = A.segP + 2 * A.cone_n * m;
        if (blockIdx.x == 0)                              // de_k += mu^{m+1}[cell_k]
            for (int k = threadIdx.x; k < A.n_src; k += blockDim.x) {
                const long long c = A.src_cell[k];
                if (c >= 0 && c < (long long)A.cells) {
                    const DF v = mu_load(Yin, Xin, A.cells, (size_t)c);
                    A.de[k] += (double)v.hi + (double)v.lo;
                }
            }
        float tD = 0.f, tL = 0.f;
        // Work per warp.  Cone warps (warp 7 of the first n_cone_warps blocks, one
        // per block so that the FP64 work spreads over many SMs: GB300's FP64 rate
        // per SM is low) take the 32-cone chunks; every other warp takes an equal
        // contiguous share of the field rows, strip by strip, so every SM gets the
        // same amount of field work.
        const int warp = threadIdx.x >> 5;
        const int bid = blockIdx.x;
        const bool cone_warp = warp == 7 && bid < A.n_cone_warps;
        for (int chunk = bid; cone_warp && chunk < A.n_chunks; chunk += A.n_cone_warps) {
            const int a = chunk * 32 + (threadIdx.x & 31);
            if (a < A.n && A.active[a]) {
                float p[2], d[2];
                double pb[2], db[2];
                for (int i = 0; i < 2; ++i) {
                    p[i] = __ldg(Pm + (size_t)i * A.n + a);
                    d[i] = __ldg(Pm + A.cone_n + (size_t)i * A.n + a);
                    pb[i] = __ldcg(A.pbar + (size_t)i * A.n + a);
                    db[i] = __ldcg(A.dbar + (size_t)i * A.n + a);
                }
                cone_adjoint2(A.f, A.c, A.inv_h64, Cm, (uint32_t)a, g, p, d, pb, db, Xout);
                for (int i = 0; i < 2; ++i) {
                    A.pbar[(size_t)i * A.n + a] = pb[i];
                    A.dbar[(size_t)i * A.n + a] = db[i];
                }
            }
        }
        if (!cone_warp) {
            const long long total = (long long)A.ntx * A.f.ny;                  // (strip, row) pairs
            const int rw = bid * 8 - min(bid, A.n_cone_warps) + warp;           // index among the row warps
            const long long r0 = total * rw / A.n_row_warps, r1 = total * (rw + 1) / A.n_row_warps;
            for (long long r = r0; r < r1;) {
                const int tx = (int)(r / A.f.ny), y = (int)(r % A.f.ny);
                const int n = (int)min(r1 - r, (long long)(A.f.ny - y));
                adj_rows(A, Yin, Xin, Yout, Xz, Cm, tx, y, y + n, tD, tL);
                r += n;
            }
        }
        sD = df_add(sD, DF{tD, 0.f});
        sL = df_add(sL, DF{tL, 0.f});
        if (!grid_barrier(bar, expected, limit, status)) return;
    }
    block_add2<true>(sD.hi, sL.hi, A.part);
    block_add2<true>(sD.lo, sL.lo, A.part);
}

// One backward step of the cones (+ de_k += mu_in[cell_k] by the first threads).
template <int DIM>
__global__ void __launch_bounds__(256) adj_cone_kernel(FieldDesc f, ConeDesc c, const float *__restrict__ C,
                                                       uint32_t step, int n, const float *__restrict__ P,
                                                       const float *__restrict__ Dd,
                                                       const uint8_t *__restrict__ active, double *pbar,
                                                       double *dbar, float *mu_out, const float *__restrict__ mu_in,
                                                       const int32_t *__restrict__ src_cell, int n_src,
                                                       double *de_acc)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n_src) {
        const long long cell = src_cell[a];
        const long long n_cells = (long long)f.nx * f.ny * f.nz;
        if (cell >= 0 && cell < n_cells) de_acc[a] += (double)mu_in[cell] + (double)mu_in[n_cells + cell];
    }
    if (a >= n || !active[a]) return;
    float p[DIM], d[DIM];
    double pb[DIM], db[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        p[i] = P[(size_t)i * n + a];
        d[i] = Dd[(size_t)i * n + a];
        pb[i] = pbar[(size_t)i * n + a];
        db[i] = dbar[(size_t)i * n + a];
    }
    const double inv_hd = 1.0 / (double)f.h;
    if constexpr (DIM == 2)
        cone_adjoint2(f, c, inv_hd, C, (uint32_t)a, step, p, d, pb, db, mu_out);
    else
        cone_adjoint3(f, c, inv_hd, C, (uint32_t)a, step, p, d, pb, db, mu_out);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        pbar[(size_t)i * n + a] = pb[i];
        dbar[(size_t)i * n + a] = db[i];
    }
}

// Loss and dL/dp^T = 2 (p^T - t)/n, dL/dd^T = 0.
__global__ void __launch_bounds__(256) adj_loss_kernel(int n, int dim, const float *__restrict__ P,
                                                       const float *__restrict__ T, double *pbar, double *dbar,
                                                       double *loss_acc)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    float s = 0.0f;
    if (a < n) {
        for (int i = 0; i < dim; ++i) {
            const float e = P[(size_t)i * n + a] - T[(size_t)i * n + a];
            s = fmaf(e, e, s);
            pbar[(size_t)i * n + a] = 2.0 * (double)e / (double)n;
            dbar[(size_t)i * n + a] = 0.0;
        }
    }
    block_add2<false>(s, 0.0f, loss_acc);
}

// The endpoint loss alone, L = (1/n) sum_a |p_a - t_a|^2, by one block:
// per-thread FP32 sums over a grid-stride share of the cones, block total in
// FP64, written as FP32 (no accumulator left behind in device memory).
__global__ void __launch_bounds__(1024) loss_only_kernel(int n, int dim, const float *__restrict__ P,
                                                         const float *__restrict__ T, float *out)
{
    __shared__ double sw[32];
    float s = 0.0f;
    for (int a = threadIdx.x; a < n; a += blockDim.x)
        for (int i = 0; i < dim; ++i) {
            const float e = P[(size_t)i * n + a] - T[(size_t)i * n + a];
            s = fmaf(e, e, s);
        }
    double v = warp_sum((double)s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sw[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sw[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) *out = n > 0 ? (float)(v / (double)n) : 0.0f;
    }
}

// Scale the accumulators into the caller's outputs (block 0 sums the field
// kernel's per-block dD / dlambda slots).
__global__ void __launch_bounds__(256) adj_finalize_kernel(FieldDesc f, int n_axons, const double *acc, int n_src,
                                                           const double *part, int n_part, float *gD, float *gl,
                                                           float *gsrc, float *loss, const double *S, float *gmap,
                                                           size_t n_cells)
{
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (blockIdx.x == 0) {
        __shared__ double sd[256], sl[256];
        double d = 0.0, l = 0.0;
        for (int i = threadIdx.x; i < n_part; i += blockDim.x) {
            d += part[2 * i];
            l += part[2 * i + 1];
        }
        sd[threadIdx.x] = d;
        sl[threadIdx.x] = l;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) {
                sd[threadIdx.x] += sd[threadIdx.x + w];
                sl[threadIdx.x] += sl[threadIdx.x + w];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            *gD = (float)((double)f.dt / ((double)f.h * f.h) * sd[0]);
            *gl = (float)(-(double)f.dt * sl[0]);
            *loss = (float)(acc[2 + n_src] / (n_axons > 0 ? n_axons : 1));
        }
    }
    if (t < (size_t)n_src) gsrc[t] = (float)acc[2 + t];
    if (gmap)
        for (size_t c = t; c < n_cells; c += (size_t)gridDim.x * blockDim.x) gmap[c] = (float)((double)f.dt * S[c]);
}

struct AdjLayout {
    size_t ckpt_c, ckpt_p, seg_c, seg_p, mu, Sseg, S, pbar, acc, part, bar, total;
    int n_part;
    int nseg;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int blocks_for(size_t n, int per) { return (int)((n + per - 1) / per); }

constexpr int kAdjMaxBlocksPerSm = 8;

int sm_count_adj()
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

// Launch shape of the backward field kernel: the float4 kernel's (x blocks,
// y blocks, rows) for 2D grids with nx % 4 == 0, else a 1D grid.  The layout
// reserves one (dD, dlambda) slot pair per block.
struct AdjFieldShape {
    bool vec4;
    int xb, yb, rows, blocks;
};

AdjFieldShape adj_field_shape(const cue_params &p)
{
    AdjFieldShape g{};
    const size_t cells = (size_t)p.nx * p.ny * (p.dim == 3 ? p.nz : 1);
    g.vec4 = p.dim == 2 && p.nx % 4 == 0;
    if (g.vec4) {
        const int BY = 8;
        g.xb = (p.nx / 4 + 31) / 32;
        g.rows = 8;      // the most rows per thread that still leaves >= 4 blocks per SM
        while (g.rows > 1 && (long long)g.xb * ((p.ny + BY * g.rows - 1) / (BY * g.rows)) < 4LL * sm_count_adj())
            g.rows /= 2;
        g.yb = (p.ny + BY * g.rows - 1) / (BY * g.rows);
        g.blocks = g.xb * g.yb;
    } else {
        g.blocks = std::min(blocks_for(cells, 256), sm_count_adj() * 16);
    }
    return g;
}

int adj_field_blocks(const cue_params &p) { return adj_field_shape(p).blocks; }

AdjLayout adj_layout(const cue_params &p, int n_src, int n_axons, int nsteps, int k)
{
    AdjLayout L{};
    const size_t cells = (size_t)p.nx * p.ny * (p.dim == 3 ? p.nz : 1);
    const size_t cone = (size_t)2 * p.dim * (n_axons > 0 ? n_axons : 1);    // pos + dir
    L.nseg = (nsteps + k - 1) / k;
    size_t off = 0;
    L.ckpt_c = off;                               // checkpoints of every segment but the last
    off += align256(sizeof(float) * cells * (L.nseg - 1));
    L.ckpt_p = off;
    off += align256(sizeof(float) * cone * (L.nseg - 1));
    const size_t seg_states = (size_t)std::min(k, nsteps) + 1;
    L.seg_c = off;
    off += align256(sizeof(float) * cells * seg_states);
    L.seg_p = off;
    off += align256(sizeof(float) * cone * seg_states);
    L.mu = off;                                   // adjoint field: five double-float buffers (hi, lo planes):
    off += align256(sizeof(float) * cells * 10);  // Y[2] and X[3] of the persistent backward, or mu[2]
    L.Sseg = off;                                 // this segment's sum of mu (double-float: hi, lo planes)
    off += align256(sizeof(float) * cells * 2);
    L.S = off;                                    // FP64 sum over the segments (rate-map gradient)
    off += align256(sizeof(double) * cells);
    L.pbar = off;
    off += align256(sizeof(double) * cone);        // dL/dp and dL/dd, FP64
    L.acc = off;                                  // spare, spare, de[n_src], loss, spare
    off += align256(sizeof(double) * (4 + n_src));
    L.n_part = std::max(adj_field_blocks(p), kAdjMaxBlocksPerSm * sm_count_adj());
    L.part = off;                                 // per-block (dD, dlambda) sums of the field kernel
    off += align256(sizeof(double) * 2 * (size_t)L.n_part);
    L.bar = off;                                  // grid barrier of the persistent backward
    off += 256;
    L.total = off;
    return L;
}

int adj_persist_blocks_per_sm()
{
    static int nb = -1;
    if (nb < 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, adj_persist_kernel, 256, 0) != cudaSuccess) v = 0;
        nb = std::min(v, kAdjMaxBlocksPerSm);
    }
    return nb;
}

bool adj_persist_supported(const Sim &s)
{
    return s.path != CUE_PATH_PLAIN && s.fd.dim == 2 && s.fd.nx % 4 == 0 && adj_persist_blocks_per_sm() > 0;
}

void launch_adj_field(Sim &s, const float *mu_in, float *mu_out, const float *C, float *Sseg, double *acc)
{
    const FieldDesc &f = s.fd;
    const size_t cells = (size_t)f.nx * f.ny * f.nz;
    const bool aligned = ((reinterpret_cast<uintptr_t>(mu_in) | reinterpret_cast<uintptr_t>(mu_out) |
                           reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(Sseg)) & 15u) == 0;
    const AdjFieldShape g = adj_field_shape(s.params);
    if (g.vec4 && aligned) {
        adj_field2d_vec4<<<dim3(g.xb, g.yb), dim3(32, 8), 0, s.stream>>>(f, mu_in, mu_out, C, Sseg, acc, g.rows);
    } else {
        adj_field_scalar<<<std::min(g.blocks, blocks_for(cells, 256)), 256, 0, s.stream>>>(f, mu_in, mu_out, C,
                                                                                           Sseg, acc);
    }
    s.launches++;
}

}  // namespace

cudaError_t launch_endpoint_loss(Sim &s, const float *targets, float *loss)
{
    loss_only_kernel<<<1, 1024, 0, s.stream>>>(s.n_axons, s.fd.dim, s.pos, targets, loss);
    s.launches++;
    return cudaGetLastError();
}

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
    float *mu[2] = {reinterpret_cast<float *>(W + L.mu), reinterpret_cast<float *>(W + L.mu) + 2 * cells};
    float *Sseg = gmap ? reinterpret_cast<float *>(W + L.Sseg) : nullptr;
    double *S = gmap ? reinterpret_cast<double *>(W + L.S) : nullptr;
    double *pbar = reinterpret_cast<double *>(W + L.pbar), *dbar = pbar + cone_n;
    double *acc = reinterpret_cast<double *>(W + L.acc);     // spare, spare, de[n_src], loss
    double *part = reinterpret_cast<double *>(W + L.part);   // per-block (dD, dlambda) sums
    cudaStream_t st = s.stream;
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    if (!ok(cudaMemsetAsync(mu[0], 0, sizeof(float) * cells * 10, st)) ||
        !ok(cudaMemsetAsync(acc, 0, sizeof(double) * (4 + s.n_src), st)) ||
        !ok(cudaMemsetAsync(part, 0, sizeof(double) * 2 * (size_t)L.n_part, st)) ||
        (S && !ok(cudaMemsetAsync(S, 0, sizeof(double) * cells, st))) ||
        (Sseg && !ok(cudaMemsetAsync(Sseg, 0, sizeof(float) * cells * 2, st))))
        return CUE_ERR_CUDA;
    const int64_t n0 = s.field_step;
    // one segment's coupled steps storing every state in sgC / sgP (slot 0 holds
    // its start): one persistent launch where the path runs, else a cone and a
    // field launch per step
    auto trajectory = [&](int len, int64_t nstart) -> int {
        int rc = (s.path != CUE_PATH_PLAIN && persist_supported(s))
                     ? run_persist_trajectory(s, sgC, sgP, (uint32_t)nstart, len)
                     : 1;
        if (rc < 0) return rc;
        for (int m = 0; rc == 1 && m < len; ++m) {
            float *Pm = sgP + 2 * cone_n * m, *Pn = sgP + 2 * cone_n * (m + 1);
            if (!ok(launch_cone_step_io(s, sgC + cells * m, (uint32_t)(nstart + m), Pm, Pm + cone_n, Pn,
                                        Pn + cone_n)) ||
                !ok(launch_field_and_sources(s, sgC + cells * m, sgC + cells * (m + 1))))
                return CUE_ERR_CUDA;
        }
        return CUE_OK;
    };
    // ---- forward: checkpoints every k steps on the fastest path; the last segment
    // runs as a stored trajectory, which its backward then walks without a
    // recompute (with k >= nsteps the whole run is one stored trajectory and
    // nothing is recomputed)
    for (int j = 0; j < L.nseg - 1; ++j) {
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
    {
        const int jl = L.nseg - 1;
        const int len = nsteps - jl * k;
        if (!ok(cudaMemcpyAsync(sgC, s.field[s.cur], sizeof(float) * cells, cudaMemcpyDeviceToDevice, st)) ||
            !ok(cudaMemcpyAsync(sgP, s.pos, sizeof(float) * cone_n, cudaMemcpyDeviceToDevice, st)) ||
            !ok(cudaMemcpyAsync(sgP + cone_n, s.dir, sizeof(float) * cone_n, cudaMemcpyDeviceToDevice, st)))
            return CUE_ERR_CUDA;
        int rc = trajectory(len, n0 + (int64_t)jl * k);
        if (rc != CUE_OK) return rc;
        // the handle ends as after sim_run: C^T in the buffer that is then current,
        // C^{T-1} in the other, the cones at step T
        const int cur_end = s.cur ^ (len & 1);
        if (!ok(cudaMemcpyAsync(s.field[cur_end], sgC + cells * len, sizeof(float) * cells,
                                cudaMemcpyDeviceToDevice, st)) ||
            !ok(cudaMemcpyAsync(s.field[cur_end ^ 1], sgC + cells * (len - 1), sizeof(float) * cells,
                                cudaMemcpyDeviceToDevice, st)) ||
            !ok(cudaMemcpyAsync(s.pos, sgP + 2 * cone_n * len, sizeof(float) * cone_n, cudaMemcpyDeviceToDevice,
                                st)) ||
            !ok(cudaMemcpyAsync(s.dir, sgP + 2 * cone_n * len + cone_n, sizeof(float) * cone_n,
                                cudaMemcpyDeviceToDevice, st)))
            return CUE_ERR_CUDA;
        s.cur = cur_end;
        s.field_step += len;
        s.cone_step += len;
    }
    // ---- loss and its adjoint at the end
    if (n > 0) {
        adj_loss_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, dim, s.pos, targets, pbar, dbar, acc + 2 + s.n_src);
        s.launches++;
    }
    // ---- backwards through the segments: one persistent launch per segment where
    // the path runs (2D, nx % 4 == 0), else two launches per step
    const bool persist_bw = adj_persist_supported(s);
    AdjP A{};
    int bw_grid = 0;
    if (persist_bw) {
        A.f = f;
        A.c = s.cd;
        A.inv_h64 = 1.0 / (double)f.h;
        A.n = n;
        A.n_src = s.n_src;
        A.src_cell = s.src_cell;
        A.active = s.active;
        A.pbar = pbar;
        A.dbar = dbar;
        A.cells = cells;
        A.cone_n = cone_n;
        float *base = reinterpret_cast<float *>(W + L.mu);
        A.Y[0] = base;
        A.Y[1] = base + 2 * cells;
        for (int i = 0; i < 3; ++i) A.X[i] = base + (4 + 2 * i) * cells;
        A.Sseg = Sseg;
        A.part = part;
        A.de = acc + 2;
        A.ntx = (f.nx / 4 + 31) / 32;
        A.n_chunks = blocks_for((size_t)n, 32);
        bw_grid = std::max(1, std::min(2, adj_persist_blocks_per_sm()) * sm_count_adj());
        A.n_cone_warps = std::min(A.n_chunks, bw_grid);
        A.n_row_warps = bw_grid * 8 - A.n_cone_warps;
    }
    int in = 0;
    for (int j = L.nseg - 1; j >= 0; --j) {
        const int len = std::min(k, nsteps - j * k);
        const int64_t nstart = n0 + (int64_t)j * k;
        if (j < L.nseg - 1) {         // recompute the segment from its checkpoint, storing every step
            if (!ok(cudaMemcpyAsync(sgC, ckC + cells * j, sizeof(float) * cells, cudaMemcpyDeviceToDevice, st)) ||
                !ok(cudaMemcpyAsync(sgP, ckP + 2 * cone_n * j, sizeof(float) * 2 * cone_n, cudaMemcpyDeviceToDevice,
                                    st)))
                return CUE_ERR_CUDA;
            int rc = trajectory(len, nstart);
            if (rc != CUE_OK) return rc;
        }
        if (s.adj_trace_field &&
            (!ok(cudaMemcpyAsync(s.adj_trace_field + cells * (size_t)j * k, sgC, sizeof(float) * cells * (len + 1),
                                 cudaMemcpyDeviceToDevice, st)) ||
             !ok(cudaMemcpyAsync(s.adj_trace_cone + 2 * cone_n * (size_t)j * k, sgP,
                                 sizeof(float) * 2 * cone_n * (len + 1), cudaMemcpyDeviceToDevice, st))))
            return CUE_ERR_CUDA;
        if (persist_bw) {
            A.segC = sgC;
            A.segP = sgP;
            if (!ok(cudaMemsetAsync(W + L.bar, 0, 256, st))) return CUE_ERR_CUDA;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(bw_grid);
            cfg.blockDim = dim3(256);
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (!ok(cudaLaunchKernelEx(&cfg, adj_persist_kernel, A, len, (uint32_t)nstart,
                                       reinterpret_cast<PBar *>(W + L.bar), (unsigned)bw_grid, kPersistSpinLimit,
                                       s.status())))
                return CUE_ERR_CUDA;
            s.launches++;
        }
        for (int m = len - 1; !persist_bw && m >= 0; --m) {
            const float *Cm = sgC + cells * m, *Pm = sgP + 2 * cone_n * m;
            launch_adj_field(s, mu[in], mu[in ^ 1], Cm, Sseg, part);
            const int cb = blocks_for((size_t)std::max(n, s.n_src), 32);   // FP64 work: many SMs
            if (cb > 0) {
                if (dim == 2)
                    adj_cone_kernel<2><<<cb, 32, 0, st>>>(f, s.cd, Cm, (uint32_t)(nstart + m), n, Pm, Pm + cone_n,
                                                           s.active, pbar, dbar, mu[in ^ 1], mu[in], s.src_cell,
                                                           s.n_src, acc + 2);
                else
                    adj_cone_kernel<3><<<cb, 32, 0, st>>>(f, s.cd, Cm, (uint32_t)(nstart + m), n, Pm, Pm + cone_n,
                                                           s.active, pbar, dbar, mu[in ^ 1], mu[in], s.src_cell,
                                                           s.n_src, acc + 2);
                s.launches++;
            }
            if (!ok(cudaGetLastError())) return CUE_ERR_CUDA;
            in ^= 1;
        }
        if (S) {
            adj_fold_kernel<<<std::min(blocks_for(cells, 256), 152 * 8), 256, 0, st>>>(cells, Sseg, S);
            s.launches++;
        }
    }
    adj_finalize_kernel<<<std::max(blocks_for((size_t)s.n_src, 256), std::min(blocks_for(cells, 256), 152 * 8)),
                          256, 0, st>>>(
        f, n, acc, s.n_src, part, L.n_part, gD, gl, gsrc, loss, S, gmap, cells);
    s.launches++;
    return ok(cudaGetLastError()) ? CUE_OK : CUE_ERR_CUDA;
}

}  // namespace cue
