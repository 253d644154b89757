// k_resident.cu -- small 2D grids held in one block's shared memory for a
// whole call.
//
// When both buffers of a 2D field fit in shared memory (a 128^2 grid takes
// 128 KB), one 1024-thread block keeps them there for every step of a call:
// the first warps update the field from one buffer into the other, the last
// warps each carry 32 growth cones in registers and step them on the same
// buffer, and one __syncthreads per step separates the steps.  Global memory
// is read at the start (field, sources, cone state) and written at the end
// (both buffers, cone state), so a step costs one pass of one SM over shared
// memory, not a pass through L2 and a grid-wide barrier.
//
// The SM issues every instruction of a step, so the field loop is built to
// issue few: a warp takes a band of `rows` rows of a 128-column block (a lane
// per four columns), keeps the rows above, at and below in registers and
// loads one new row per row it updates; its x neighbours come from the
// adjacent lanes; a per-row bitmap in shared memory sends only the rows that
// hold a source through the source list.
//
// Per node and per cone the arithmetic is the plain path's: node_update2, the
// rate map as fma(dt, M, C'), the point sources added after that in source
// order, and cone_step_rule on C^n.  Results therefore agree with the plain
// and persistent paths bit for bit (for distinct source cells).  There is no
// wait in the kernel other than __syncthreads.
#include <algorithm>

#include "cue_internal.h"

namespace cue {
namespace {

constexpr unsigned kFullR = 0xffffffffu;

struct ResArgs {
    FieldDesc f;
    ConeDesc c;
    const float *Cin;            // C^n, dense rows of nx floats
    float *Cout;                 // receives C^{n+k}
    float *Cprev;                // receives C^{n+k-1} (the other buffer)
    const float *map;            // rate map (same layout) or null
    const int32_t *src_cell;
    const float *src_emit;
    const float *src_xyz;        // [2][n_src] source coordinates for the stop test
    int n_src;
    float *pos, *dir;            // [2][n_axons]
    uint8_t *active;
    int n_axons;
    int nsteps;
    uint32_t step0;              // Philox step of the first step
    int field_warps;             // warps 0 .. field_warps-1 update the field; the rest step cones
    int rows;                    // rows per band of the field loop
    unsigned *status;
    unsigned long long *counter;
};

__device__ __forceinline__ bool finite4r(const float4 &v)
{
    const float big = 3.402823466e38f;
    return fabsf(v.x) <= big && fabsf(v.y) <= big && fabsf(v.z) <= big && fabsf(v.w) <= big;
}

// Bits of rows y .. y + 31 from the per-row source bitmap (bit i: row y + i holds a source).
__device__ __forceinline__ unsigned row_bits(const unsigned *rows, int nrw, int y)
{
    const int w = y >> 5;
    const unsigned lo = rows[w], hi = w + 1 < nrw ? rows[w + 1] : 0u;
    return __funnelshift_r(lo, hi, y & 31);
}

template <bool MAP>
__global__ void __launch_bounds__(kResThreads, 1) resident_kernel(const __grid_constant__ ResArgs A)
{
    extern __shared__ __align__(16) float smem[];
    const FieldDesc &f = A.f;
    const int nx = f.nx, ny = f.ny;
    const float alpha = f.alpha, beta = f.beta, dt = f.dt;
    const int cells = nx * ny;                        // a multiple of 4 (nx % 4 == 0)
    const int nq = cells >> 2;                        // float4 groups
    const int Q = nx >> 2;                            // float4 groups per row
    const int nrw = (ny + 31) >> 5;                   // words of the per-row source bitmap
    float *buf0 = smem, *buf1 = smem + cells;
    int *s_cell = reinterpret_cast<int *>(smem + 2 * cells);
    float *s_emit = smem + 2 * cells + A.n_src;
    unsigned *s_rows = reinterpret_cast<unsigned *>(smem + 2 * cells + 2 * A.n_src);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // C^n and the sources into shared memory (cells outside the grid are
    // reported and left out), then the rows that hold a source
    {
        const float4 *in4 = reinterpret_cast<const float4 *>(A.Cin);
        float4 *b4 = reinterpret_cast<float4 *>(buf0);
        for (int q = tid; q < nq; q += kResThreads) b4[q] = __ldg(in4 + q);
        for (int k = tid; k < A.n_src; k += kResThreads) {
            int c = __ldg(A.src_cell + k);
            if (c < 0 || c >= cells) {
                flag_status(A.status, kStatusBounds);
                c = -1;
            }
            s_cell[k] = c;
            s_emit[k] = __ldg(A.src_emit + k);
        }
        for (int w = tid; w < nrw; w += kResThreads) s_rows[w] = 0u;
    }
    __syncthreads();
    for (int k = tid; k < A.n_src; k += kResThreads) {
        const int c = s_cell[k];
        if (c >= 0) {
            const int y = c / nx;
            atomicOr(s_rows + (y >> 5), 1u << (y & 31));
        }
    }
    __syncthreads();

    const bool field_warp = warp < A.field_warps;
    // the field loop's work items: column blocks of 32 groups x bands of `rows` rows
    const int ncb = (Q + 31) >> 5;
    const int R = A.rows;
    const int n_items = ncb * ((ny + R - 1) / R);

    // cone state of this lane, in registers for the whole call
    const int a = (warp - A.field_warps) * 32 + lane;
    const bool has_cone = !field_warp && a < A.n_axons;
    float p[2] = {0.f, 0.f}, d[2] = {0.f, 0.f};
    bool act = false;
    if (has_cone) {
        p[0] = A.pos[a];
        p[1] = A.pos[A.n_axons + a];
        d[0] = A.dir[a];
        d[1] = A.dir[A.n_axons + a];
        act = A.active[a] != 0;
    }
    const bool stop = A.c.stop_r2 >= 0.0f && A.n_src > 0;
    unsigned n_live = 0;
    bool bad = false;

    float *cur = buf0, *nxt = buf1;
    for (int s = 0; s < A.nsteps; ++s) {
        if (field_warp) {
            const float4 *c4 = reinterpret_cast<const float4 *>(cur);
            float4 *o4 = reinterpret_cast<float4 *>(nxt);
            for (int it = warp; it < n_items; it += A.field_warps) {    // warp-uniform
                const int cb = it % ncb, y0 = (it / ncb) * R, y1 = min(y0 + R, ny);
                const int x4 = cb * 32 + lane;        // this lane's group in the row
                const bool xin = x4 < Q;
                const bool need_l = lane == 0 && x4 > 0, need_r = lane == 31 && x4 + 1 < Q;
                const bool wall_l = x4 == 0, wall_r = x4 + 1 >= Q;
                // lanes past the right edge read the last group and drop their results
                const float4 *col = c4 + (xin ? x4 : Q - 1);
                // rows y - 1 and y + 1 are read clamped: at a wall they are row y itself
                float4 vm = col[max(y0 - 1, 0) * Q];
                float4 vc = col[y0 * Q];
                unsigned bits = 0;
#pragma unroll 4
                for (int y = y0; y < y1; ++y) {
                    const float4 vp = col[(y + 1 < ny ? y + 1 : y) * Q];
                    if (((y - y0) & 31) == 0) bits = row_bits(s_rows, nrw, y);
                    float l = __shfl_up_sync(kFullR, vc.w, 1);
                    float r = __shfl_down_sync(kFullR, vc.x, 1);
                    if (need_l) l = cur[y * nx + 4 * x4 - 1];
                    if (need_r) r = cur[y * nx + 4 * x4 + 4];
                    if (wall_l) l = vc.x;             // a wall: the missing neighbour is the node itself
                    if (wall_r) r = vc.w;
                    float4 o;
                    o.x = node_update2(vc.x, l, vc.y, vm.x, vp.x, alpha, beta);
                    o.y = node_update2(vc.y, vc.x, vc.z, vm.y, vp.y, alpha, beta);
                    o.z = node_update2(vc.z, vc.y, vc.w, vm.z, vp.z, alpha, beta);
                    o.w = node_update2(vc.w, vc.z, r, vm.w, vp.w, alpha, beta);
                    const int q = y * Q + x4;
                    if constexpr (MAP) {
                        const float4 m = __ldg(reinterpret_cast<const float4 *>(A.map) + (xin ? q : 0));
                        o.x = fmaf(dt, m.x, o.x);
                        o.y = fmaf(dt, m.y, o.y);
                        o.z = fmaf(dt, m.z, o.z);
                        o.w = fmaf(dt, m.w, o.w);
                    }
                    if (bits & 1u) {                  // the row's sources at these nodes, in source order
                        for (int k = 0; k < A.n_src; ++k) {
                            const int rel = s_cell[k] - 4 * q;
                            if (rel >= 0 && rel < 4) {
                                const float em = s_emit[k];
                                if (rel == 0) o.x += em;
                                else if (rel == 1) o.y += em;
                                else if (rel == 2) o.z += em;
                                else o.w += em;
                            }
                        }
                    }
                    bits >>= 1;
                    if (xin) o4[q] = o;
                    vm = vc;
                    vc = vp;
                }
            }
        } else if (has_cone) {
            float xi[2];
            cone_noise<2>(A.c.key0, A.c.key1, (uint32_t)a, A.step0 + (uint32_t)s, xi);
            if (act) {
                ++n_live;
                const float *Cs = cur;
                auto ld = [&](int i, int j, int) { return Cs[i + nx * j]; };
                act = cone_step_rule<2>(f, A.c, ld, xi, p, d, A.src_xyz, A.n_src, stop ? A.n_src : 0);
                const float big = 3.402823466e38f;
                if (!(fabsf(p[0]) <= big && fabsf(p[1]) <= big && fabsf(d[0]) <= big && fabsf(d[1]) <= big))
                    bad = true;
            }
        }
        __syncthreads();
        float *t = cur;
        cur = nxt;
        nxt = t;
    }

    // cur holds C^{n+k}, nxt C^{n+k-1}; non-finite values persist, so testing the
    // last step's output covers the call
    {
        const float4 *cur4 = reinterpret_cast<const float4 *>(cur), *nxt4 = reinterpret_cast<const float4 *>(nxt);
        float4 *out4 = reinterpret_cast<float4 *>(A.Cout), *prev4 = reinterpret_cast<float4 *>(A.Cprev);
        for (int q = tid; q < nq; q += kResThreads) {
            const float4 v = cur4[q];
            bad |= !finite4r(v);
            out4[q] = v;
            prev4[q] = nxt4[q];
        }
    }
    if (has_cone) {
        A.pos[a] = p[0];
        A.pos[A.n_axons + a] = p[1];
        A.dir[a] = d[0];
        A.dir[A.n_axons + a] = d[1];
        A.active[a] = act ? 1 : 0;
    }
    if (__any_sync(kFullR, bad) && lane == 0) flag_status(A.status, kStatusNonFinite);
    if (!field_warp) {                                // warp-uniform
        const unsigned tot = __reduce_add_sync(kFullR, n_live);
        if (lane == 0 && tot) atomicAdd(A.counter, (unsigned long long)tot);
    }
}

size_t resident_smem_bytes(const Sim &s)
{
    return 2 * sizeof(float) * (size_t)s.fd.nx * s.fd.ny + 8 * (size_t)s.n_src + 4 * (size_t)((s.fd.ny + 31) / 32);
}

int resident_smem_limit()
{
    static int limit = -1;
    if (limit < 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 0;
        limit = v;
    }
    return limit;
}

}  // namespace

bool resident_supported(const Sim &s)
{
    return s.fd.dim == 2 && s.vec4 && s.n_axons <= kResMaxCones && s.n_src <= kResMaxSources &&
           resident_smem_bytes(s) <= (size_t)resident_smem_limit();
}

int run_resident_if_supported(Sim &s, int nsteps)
{
    if (s.path != CUE_PATH_AUTO && s.path != CUE_PATH_RESIDENT) return 1;
    if (!resident_supported(s)) return s.path == CUE_PATH_RESIDENT ? CUE_ERR_ARG : 1;
    if (nsteps <= 0) return CUE_OK;
    if (s.cd.stop_r2 >= 0.0f && s.n_src > 0 && !s.src_xyz_ready) {
        if (launch_src_xyz(s) != cudaSuccess) return CUE_ERR_CUDA;
        s.src_xyz_ready = true;
    }
    const size_t smem = resident_smem_bytes(s);
    const bool map = s.src_map != nullptr;
    // the shared-memory allowance is a per-device function attribute: set it
    // once on every device this process launches the kernel on
    static unsigned long long attr_set[2] = {0ull, 0ull};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CUE_ERR_CUDA;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!(attr_set[map] & bit)) {
        cudaError_t e = map ? cudaFuncSetAttribute(resident_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   resident_smem_limit())
                            : cudaFuncSetAttribute(resident_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   resident_smem_limit());
        if (e != cudaSuccess) return CUE_ERR_CUDA;
        attr_set[map] |= bit;
    }
    ResArgs A{};
    A.f = s.fd;
    A.c = s.cd;
    A.map = s.src_map;
    A.src_cell = s.src_cell;
    A.src_emit = s.src_emit;
    A.src_xyz = s.src_xyz();
    A.n_src = s.n_src;
    A.pos = s.pos;
    A.dir = s.dir;
    A.active = s.active;
    A.n_axons = s.n_axons;
    A.field_warps = kResThreads / 32 - (s.n_axons + 31) / 32;
    // bands just tall enough that every field warp has at most one work item
    const int ncb = (s.fd.nx / 4 + 31) / 32;
    A.rows = std::max(1, (s.fd.ny * ncb + A.field_warps - 1) / A.field_warps);
    A.status = s.status();
    A.counter = s.cone_counter();
    for (int done = 0; done < nsteps;) {              // launches of at most kPersistMaxSteps steps
        const int k = std::min(nsteps - done, kPersistMaxSteps);
        A.Cin = s.field[s.cur];
        A.Cout = s.field[s.cur ^ (k & 1)];
        A.Cprev = s.field[s.cur ^ (k & 1) ^ 1];
        A.nsteps = k;
        A.step0 = (uint32_t)s.cone_step;
        timing_begin(s);
        if (map)
            resident_kernel<true><<<1, kResThreads, smem, s.stream>>>(A);
        else
            resident_kernel<false><<<1, kResThreads, smem, s.stream>>>(A);
        timing_end(s);
        s.launches++;
        if (cudaGetLastError() != cudaSuccess) return CUE_ERR_CUDA;
        s.cur ^= (k & 1);
        s.field_step += k;
        s.cone_step += k;
        done += k;
    }
    s.resident_used = true;
    return CUE_OK;
}

}  // namespace cue
