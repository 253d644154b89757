// cue_device.cuh -- device-side building blocks shared by the CUDA kernels of
// libcue.so: parameter blocks, the Philox-4x32-10 counter generator, the
// Box-Muller noise, multilinear gradient sampling and the growth-cone update.
//
// Model: Mihut, Morgan & Kaiser, cue diffusion on an Eulerian grid (Sec. 5.2)
// steering growth cones by vector addition of the current direction and the
// sensed cue direction (Sec. 3.5, Eq. 6-7), with Gaussian noise from a
// stateless per-thread counter-based generator (Sec. 5.1) through Box-Muller
// (Sec. 3.2), and stop tests on the simulation bounds (Sec. 3.4) and on
// squared distances to the sources (Sec. 3.3).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cue {

// Field physics, precomputed on the host in FP32.
struct FieldDesc {
    int dim;
    int nx, ny, nz;     // nz == 1 in 2D
    float h;
    float alpha;        // D dt / h^2
    float decay;        // lambda dt
    float dt;
    float beta;         // 1 - 2 dim alpha - lambda dt
    float inv_h;        // 1 / h
};

// The node update used by every field kernel:
//   C' = beta C + alpha (sum of the axis neighbours),
// where a neighbour missing at a wall is replaced by the node itself, so its
// flux term alpha (C_j - C_i) vanishes (no-flux).  Neighbours are summed as
// ((x- + x+) + (y- + y+)) [+ (z- + z+)] in every kernel so that all paths
// round identically.
__device__ __forceinline__ float node_update2(float c, float xm, float xp, float ym, float yp,
                                              float alpha, float beta)
{
    return fmaf(alpha, (xm + xp) + (ym + yp), beta * c);
}

__device__ __forceinline__ float node_update3(float c, float xm, float xp, float ym, float yp,
                                              float zm, float zp, float alpha, float beta)
{
    return fmaf(alpha, ((xm + xp) + (ym + yp)) + (zm + zp), beta * c);
}

// node_update3 on a float4 group, two nodes at a time with the packed FP32x2
// instructions (each half of a pair rounds exactly like the scalar form):
// ((x- + x+) + (y- + y+)) + (z- + z+), times alpha, plus beta c.
__device__ __forceinline__ float4 node_update3_x4(const float4 &c, float xl, float xr, const float4 &ym,
                                                  const float4 &yp, const float4 &zm, const float4 &zp,
                                                  float2 alpha2, float2 beta2)
{
    const float2 hx01 = __fadd2_rn(make_float2(xl, c.x), make_float2(c.y, c.z));
    const float2 hx23 = __fadd2_rn(make_float2(c.y, c.z), make_float2(c.w, xr));
    const float2 hy01 = __fadd2_rn(make_float2(ym.x, ym.y), make_float2(yp.x, yp.y));
    const float2 hy23 = __fadd2_rn(make_float2(ym.z, ym.w), make_float2(yp.z, yp.w));
    const float2 hz01 = __fadd2_rn(make_float2(zm.x, zm.y), make_float2(zp.x, zp.y));
    const float2 hz23 = __fadd2_rn(make_float2(zm.z, zm.w), make_float2(zp.z, zp.w));
    const float2 s01 = __fadd2_rn(__fadd2_rn(hx01, hy01), hz01);
    const float2 s23 = __fadd2_rn(__fadd2_rn(hx23, hy23), hz23);
    const float2 o01 = __ffma2_rn(alpha2, s01, __fmul2_rn(beta2, make_float2(c.x, c.y)));
    const float2 o23 = __ffma2_rn(alpha2, s23, __fmul2_rn(beta2, make_float2(c.z, c.w)));
    return make_float4(o01.x, o01.y, o23.x, o23.y);
}

// Cone parameters, precomputed on the host in FP32.
struct ConeDesc {
    float w_prev, w_grad, w_noise, step_len;
    float stop_r2;      // stop_radius^2; < 0 disables the source stop
    float eps2;         // grad_eps^2
    float inv2h;        // 1 / (2 h)
    float hi0, hi1, hi2; // domain upper bound per axis: (N - 1) h
    int wall_mode;      // 0 stop, 1 clamp
    uint32_t key0, key1;
    // steering rule: 0 vector addition (Sec. 3.5, Eq. 6-7); 1 the SNR turn rule (Eq. 5, 2D)
    int steer;
    float snr_gain, snr_width, snr_inv_kd, snr_cmin, snr_cmax;
    float turn_c, turn_s;   // cos and sin of the turn angle
};

// Bits of the device status word.
enum : unsigned {
    kStatusNonFinite = 1u,
    kStatusBounds = 2u,
    kStatusTimeout = 4u,
};

__device__ __forceinline__ void flag_status(unsigned *status, unsigned bits)
{
    if (status) atomicOr(status, bits);
}

// Warp-aggregated count of active cones into a 64-bit counter (one atomic per
// warp).  Must be called by all lanes of a converged warp.
__device__ __forceinline__ void count_active(unsigned long long *counter, bool active)
{
    unsigned m = __ballot_sync(0xffffffffu, active);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(counter, (unsigned long long)__popc(m));
}

// --------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds; a round
// takes the two 64-bit products of counter words 0 and 2 with the round
// multipliers, XORs their high halves with words 1 and 3 and the two key
// words, and bumps the key by the Weyl increments.
// --------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3,
                                              uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = 0xD2511F53u, b = 0xCD9E8D57u;
        uint32_t hi_a = __umulhi(a, c0), lo_a = a * c0;
        uint32_t hi_b = __umulhi(b, c2), lo_b = b * c2;
        uint32_t n0 = hi_b ^ c1 ^ k0;
        uint32_t n2 = hi_a ^ c3 ^ k1;
        c0 = n0;
        c1 = lo_b;
        c2 = n2;
        c3 = lo_a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Gaussian vector of cone `axon` at `step`: uniforms from the top 24 bits of
// the Philox words (u1, u3 in (0,1]; u2, u4 in [0,1)), Box-Muller on
// (u1,u2) for components 0,1 and on (u3,u4) for component 2.
template <int DIM>
__device__ __forceinline__ void cone_noise(uint32_t k0, uint32_t k1, uint32_t axon, uint32_t step,
                                           float xi[DIM])
{
    uint32_t w0 = axon, w1 = step, w2 = 0u, w3 = 0u;
    philox4x32_10(w0, w1, w2, w3, k0, k1);
    const float two_m24 = 5.9604644775390625e-8f;   // 2^-24
    float u1 = (float)((w0 >> 8) + 1u) * two_m24;
    float u2 = (float)(w1 >> 8) * two_m24;
    float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    xi[0] = r * c;
    xi[1] = r * s;
    if constexpr (DIM == 3) {
        float u3 = (float)((w2 >> 8) + 1u) * two_m24;
        float u4 = (float)(w3 >> 8) * two_m24;
        float r2 = sqrtf(-2.0f * logf(u3));
        xi[2] = r2 * cospif(2.0f * u4);
    }
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// --------------------------------------------------------------------------
// Gradient at point p: multilinear interpolation of node central differences
// (a missing neighbour at a wall is replaced by the node itself).  `ld(i,j,k)`
// returns C at a node inside the grid.
// --------------------------------------------------------------------------

// Cell of p (lower corner clamped to [0, N-2] per axis) and the fractional
// position inside it.
template <int DIM>
__device__ __forceinline__ void cell_of(const FieldDesc &f, const float *p, int *lo, float *fr)
{
    const int ext[3] = {f.nx, f.ny, f.nz};
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
        float s = p[ax] * f.inv_h;
        int i0 = clampi((int)floorf(s), 0, ext[ax] - 2);
        lo[ax] = i0;
        fr[ax] = s - (float)i0;
    }
}

// The 12 nodes a 2D gradient sample reads, in a fixed order: rows y0 and y1
// across x = i0-1 .. i0+2, then columns x0 and x1 at y = j0-1 and j0+2 (indices
// clamped at the walls, i.e. the ghost node is the edge node).
constexpr int kPatch2 = 12;

template <class Load>
__device__ __forceinline__ void gather2(const FieldDesc &f, const int *lo, const Load &ld, float *v)
{
    const int xm = max(lo[0] - 1, 0), x0 = lo[0], x1 = lo[0] + 1, xp = min(lo[0] + 2, f.nx - 1);
    const int ym = max(lo[1] - 1, 0), y0 = lo[1], y1 = lo[1] + 1, yp = min(lo[1] + 2, f.ny - 1);
    v[0] = ld(xm, y0, 0);
    v[1] = ld(x0, y0, 0);
    v[2] = ld(x1, y0, 0);
    v[3] = ld(xp, y0, 0);
    v[4] = ld(xm, y1, 0);
    v[5] = ld(x0, y1, 0);
    v[6] = ld(x1, y1, 0);
    v[7] = ld(xp, y1, 0);
    v[8] = ld(x0, ym, 0);
    v[9] = ld(x1, ym, 0);
    v[10] = ld(x0, yp, 0);
    v[11] = ld(x1, yp, 0);
}

// 2D gradient from the gathered nodes and the fractional position.
__device__ __forceinline__ void grad2(const ConeDesc &c, const float *v, const float *fr, float *g)
{
    const float r0m = v[0], r00 = v[1], r01 = v[2], r0p = v[3];
    const float r1m = v[4], r10 = v[5], r11 = v[6], r1p = v[7];
    const float cm0 = v[8], cm1 = v[9], cp0 = v[10], cp1 = v[11];
    const float wx[2] = {1.0f - fr[0], fr[0]};
    const float wy[2] = {1.0f - fr[1], fr[1]};
    // node gradients at the four corners (x index a, y index b)
    float gx00 = (r01 - r0m) * c.inv2h, gx10 = (r0p - r00) * c.inv2h;
    float gx01 = (r11 - r1m) * c.inv2h, gx11 = (r1p - r10) * c.inv2h;
    float gy00 = (r10 - cm0) * c.inv2h, gy10 = (r11 - cm1) * c.inv2h;
    float gy01 = (cp0 - r00) * c.inv2h, gy11 = (cp1 - r01) * c.inv2h;
    float w00 = wx[0] * wy[0], w10 = wx[1] * wy[0], w01 = wx[0] * wy[1], w11 = wx[1] * wy[1];
    g[0] = w00 * gx00 + w10 * gx10 + w01 * gx01 + w11 * gx11;
    g[1] = w00 * gy00 + w10 * gy10 + w01 * gy01 + w11 * gy11;
}

// 3D gradient: the 32 nodes of the trilinear footprint read through `ld`.
template <class Load>
__device__ __forceinline__ void grad3(const FieldDesc &f, const ConeDesc &c, const int *lo, const float *fr,
                                      const Load &ld, float *g)
{
    const int xm = max(lo[0] - 1, 0), x0 = lo[0], x1 = lo[0] + 1, xp = min(lo[0] + 2, f.nx - 1);
    const int ym = max(lo[1] - 1, 0), y0 = lo[1], y1 = lo[1] + 1, yp = min(lo[1] + 2, f.ny - 1);
    const int zm = max(lo[2] - 1, 0), z0 = lo[2], z1 = lo[2] + 1, zp = min(lo[2] + 2, f.nz - 1);
    const float wx[2] = {1.0f - fr[0], fr[0]};
    const float wy[2] = {1.0f - fr[1], fr[1]};
    const float wz[2] = {1.0f - fr[2], fr[2]};
    const int xs[2] = {x0, x1}, ys[2] = {y0, y1}, zs[2] = {z0, z1};
    const int xl[2] = {xm, x0}, xr[2] = {x1, xp};
    const int yl[2] = {ym, y0}, yr[2] = {y1, yp};
    const int zl[2] = {zm, z0}, zr[2] = {z1, zp};
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                float w = wx[a] * wy[e] * wz[b];
                float nx_ = (ld(xr[a], ys[e], zs[b]) - ld(xl[a], ys[e], zs[b])) * c.inv2h;
                float ny_ = (ld(xs[a], yr[e], zs[b]) - ld(xs[a], yl[e], zs[b])) * c.inv2h;
                float nz_ = (ld(xs[a], ys[e], zr[b]) - ld(xs[a], ys[e], zl[b])) * c.inv2h;
                gx += w * nx_;
                gy += w * ny_;
                gz += w * nz_;
            }
    g[0] = gx;
    g[1] = gy;
    g[2] = gz;
}

template <int DIM, class Load>
__device__ __forceinline__ void sample_gradient(const FieldDesc &f, const ConeDesc &c, const float *p,
                                                const Load &ld, float *g)
{
    int lo[3] = {0, 0, 0};
    float fr[3] = {0.f, 0.f, 0.f};
    cell_of<DIM>(f, p, lo, fr);
    if constexpr (DIM == 2) {
        float v[kPatch2];
        gather2(f, lo, ld, v);
        grad2(c, v, fr, g);
    } else {
        grad3(f, c, lo, fr, ld, g);
    }
}

// --------------------------------------------------------------------------
// The rest of a growth-cone step once the gradient g at p and the noise xi are
// known: vector addition, normalisation (reciprocal square roots), advance
// and stop tests.  p, d are updated
// in place; returns false when the cone stops at this step.  src_xyz holds
// source node coordinates as rows of src_stride (x row, y row, z row).
// --------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ bool cone_finish_xi(const ConeDesc &c, const float *g, const float *xi, float *p,
                                               float *d, const float *src_xyz, int src_stride, int n_src)
{
    float gn2 = 0.f;
#pragma unroll
    for (int i = 0; i < DIM; ++i) gn2 = fmaf(g[i], g[i], gn2);
    float ginv = (gn2 > c.eps2) ? rsqrtf(gn2) : 0.0f;

    float v[DIM], vn2 = 0.f;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        v[i] = c.w_prev * d[i] + c.w_grad * (g[i] * ginv) + c.w_noise * xi[i];
        vn2 = fmaf(v[i], v[i], vn2);
    }
    float dn[DIM];
    if (vn2 > 1e-30f) {
        float vinv = rsqrtf(vn2);
#pragma unroll
        for (int i = 0; i < DIM; ++i) dn[i] = v[i] * vinv;
    } else {
#pragma unroll
        for (int i = 0; i < DIM; ++i) dn[i] = d[i];
    }
    const float hi[3] = {c.hi0, c.hi1, c.hi2};
    float pn[DIM];
    bool outside = false;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        pn[i] = fmaf(c.step_len, dn[i], p[i]);
        if (pn[i] < 0.0f || pn[i] > hi[i]) {
            outside = true;
            pn[i] = pn[i] < 0.0f ? 0.0f : hi[i];
        }
    }
    if (outside && c.wall_mode == 0) return false;   // keeps p, d of this step
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        p[i] = pn[i];
        d[i] = dn[i];
    }
    if (c.stop_r2 >= 0.0f) {
        for (int s = 0; s < n_src; ++s) {
            float d2 = 0.f;
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
                float e = pn[i] - src_xyz[i * src_stride + s];
                d2 = fmaf(e, e, d2);
            }
            if (d2 <= c.stop_r2) return false;
        }
    }
    return true;
}

// --------------------------------------------------------------------------
// The SNR turn rule (Sec. 3.5, Eq. 5; 2D).  From the cell's 12-node patch: the
// cue value C at p (bilinear in the cell's four nodes, summed in the order
// (x0,y0), (x1,y0), (x0,y1), (x1,y1)) and the gradient g.  Inside the window
// [cmin, cmax]: SNR = gain * mu * sqrt(gamma / (1 + gamma)^3) * sin(theta -
// theta_NGF) with gamma = C / kd, mu = w |g| / C, sin(theta - theta_NGF) =
// (d_y g_x - d_x g_y) / |g|; the cone turns right (clockwise) by the turn
// angle when SNR + xi0 > 0 (a draw from N(SNR, 1)), else left, and the
// rotated direction is renormalised.  Outside the window the direction is
// kept.  Then the same advance and stop tests as the vector-addition rule.
// --------------------------------------------------------------------------
template <class Load>
__device__ __forceinline__ bool cone_update_snr(const FieldDesc &f, const ConeDesc &c, const Load &ld,
                                                const float *xi, float *p, float *d, const float *src_xyz,
                                                int src_stride, int n_src)
{
    int lo[3] = {0, 0, 0};
    float fr[3] = {0.f, 0.f, 0.f};
    cell_of<2>(f, p, lo, fr);
    float v[kPatch2];
    gather2(f, lo, ld, v);
    float g[2];
    grad2(c, v, fr, g);
    // every rounding written out (explicit fma / _rn operations), so the rule
    // gives the same bits in every kernel it is inlined into
    const float wx0 = __fsub_rn(1.0f, fr[0]), wx1 = fr[0], wy0 = __fsub_rn(1.0f, fr[1]), wy1 = fr[1];
    float Cp = __fmul_rn(__fmul_rn(wx0, wy0), v[1]);
    Cp = fmaf(__fmul_rn(wx1, wy0), v[2], Cp);
    Cp = fmaf(__fmul_rn(wx0, wy1), v[5], Cp);
    Cp = fmaf(__fmul_rn(wx1, wy1), v[6], Cp);
    float dn[2] = {d[0], d[1]};
    if (Cp >= c.snr_cmin && Cp <= c.snr_cmax) {
        const float gn = __fsqrt_rn(fmaf(g[0], g[0], __fmul_rn(g[1], g[1])));
        float snr = 0.0f;
        if (gn > 0.0f && Cp > 0.0f) {
            const float gamma = __fmul_rn(Cp, c.snr_inv_kd);
            const float mu = __fdiv_rn(__fmul_rn(c.snr_width, gn), Cp);
            const float sin_rel = __fdiv_rn(fmaf(d[1], g[0], -__fmul_rn(d[0], g[1])), gn);
            const float onep = __fadd_rn(1.0f, gamma);
            const float den = __fmul_rn(__fmul_rn(onep, onep), onep);
            snr = __fmul_rn(__fmul_rn(__fmul_rn(c.snr_gain, mu), __fsqrt_rn(__fdiv_rn(gamma, den))), sin_rel);
        }
        const float sn = (__fadd_rn(snr, xi[0]) > 0.0f) ? -c.turn_s : c.turn_s;   // right: clockwise
        const float r0 = fmaf(d[0], c.turn_c, -__fmul_rn(d[1], sn));
        const float r1 = fmaf(d[0], sn, __fmul_rn(d[1], c.turn_c));
        const float inv = __fdiv_rn(1.0f, __fsqrt_rn(fmaf(r0, r0, __fmul_rn(r1, r1))));
        dn[0] = __fmul_rn(r0, inv);
        dn[1] = __fmul_rn(r1, inv);
    }
    const float hi[2] = {c.hi0, c.hi1};
    float pn[2];
    bool outside = false;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        pn[i] = fmaf(c.step_len, dn[i], p[i]);
        if (pn[i] < 0.0f || pn[i] > hi[i]) {
            outside = true;
            pn[i] = pn[i] < 0.0f ? 0.0f : hi[i];
        }
    }
    if (outside && c.wall_mode == 0) return false;   // keeps p, d of this step
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        p[i] = pn[i];
        d[i] = dn[i];
    }
    if (c.stop_r2 >= 0.0f) {
        for (int s = 0; s < n_src; ++s) {
            float d2 = 0.f;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float e = pn[i] - src_xyz[i * src_stride + s];
                d2 = fmaf(e, e, d2);
            }
            if (d2 <= c.stop_r2) return false;
        }
    }
    return true;
}

// One cone step by the handle's steering rule, with the noise already drawn:
// the vector-addition rule is exactly sample_gradient + cone_finish_xi.
template <int DIM, class Load>
__device__ __forceinline__ bool cone_step_rule(const FieldDesc &f, const ConeDesc &c, const Load &ld,
                                               const float *xi, float *p, float *d, const float *src_xyz,
                                               int src_stride, int n_src)
{
    if constexpr (DIM == 2) {
        if (c.steer == 1) return cone_update_snr(f, c, ld, xi, p, d, src_xyz, src_stride, n_src);
    }
    float g[DIM];
    sample_gradient<DIM>(f, c, p, ld, g);
    return cone_finish_xi<DIM>(c, g, xi, p, d, src_xyz, src_stride, n_src);
}

// cone_finish_xi with the noise of (axon, step) drawn here.
template <int DIM>
__device__ __forceinline__ bool cone_finish(const ConeDesc &c, const float *g, uint32_t axon, uint32_t step,
                                            float *p, float *d, const float *src_xyz, int src_stride, int n_src)
{
    float xi[DIM];
    cone_noise<DIM>(c.key0, c.key1, axon, step, xi);
    return cone_finish_xi<DIM>(c, g, xi, p, d, src_xyz, src_stride, n_src);
}

// One whole growth-cone step (gradient, then cone_finish).
template <int DIM, class Load>
__device__ __forceinline__ bool cone_update(const FieldDesc &f, const ConeDesc &c, const Load &ld,
                                            uint32_t axon, uint32_t step, float *p, float *d,
                                            const float *src_xyz, int src_stride, int n_src)
{
    float g[DIM];
    sample_gradient<DIM>(f, c, p, ld, g);
    return cone_finish<DIM>(c, g, axon, step, p, d, src_xyz, src_stride, n_src);
}

}  // namespace cue
