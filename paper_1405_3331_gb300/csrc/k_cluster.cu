// k_cluster.cu -- small 2D grids spread over a thread-block cluster for a
// whole call.
//
// One cluster of G CTAs (G = 16 where the device can schedule it, else 8; one
// CTA per SM) holds the field in distributed shared memory: CTA r owns a band
// of rows, kept in its shared memory in two buffers with one halo row above
// and below.  Each CTA is laid out like the single-SM resident kernel
// (k_resident.cu): 1024 threads, the first warps update the band (a warp
// streams a run of rows of a 128-column block, the rows above, at and below in
// registers, x neighbours by warp shuffle, a per-row bitmap sending only rows
// with a source through the band's source list), the last warps each step 32
// of the CTA's cones on the same buffer.  A warp that computes a band's first
// or last row also stores it into the neighbouring CTA's halo row of the new
// buffer (a distributed shared memory store; at a wall, into its own halo,
// which makes the edge node its own missing neighbour), so a step is one pass
// and one cluster barrier, whose release / acquire orders those stores before
// the next step reads them.  A cone's 12-node patch may lie in another CTA's
// band: those nodes are read from that CTA's shared memory.  Global memory is
// read at the start (field, sources, cone state) and written at the end (both
// buffers, cone state).
//
// Per node and per cone the arithmetic is the plain path's: node_update2, the
// rate map as fma(dt, M, C'), the point sources added after that in source
// order, and cone_step_rule on C^n -- so the results agree with the plain,
// persistent and resident paths bit for bit (for distinct source cells).
// Model: cue field on an Eulerian grid (Sec. 5.2) with sources of their own
// rates (Sec. 4.3); cone steering by vector addition (Sec. 3.5, Eq. 6-7) with
// stateless counter-based noise (Sec. 5.1, Sec. 3.2); stop tests (Sec. 3.3-3.4).
#include <cooperative_groups.h>

#include <algorithm>

#include "cue_internal.h"

namespace cue {
namespace {

namespace cg = cooperative_groups;

constexpr unsigned kFullC = 0xffffffffu;

struct ClusterArgs {
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
    int band;                    // rows per CTA (the last CTAs may own fewer, or none)
    int field_warps;             // warps 0 .. field_warps-1 update the band; the rest step cones
    int pre_noise;               // 1: field warps without rows draw the cones' noise a step ahead
    int rows;                    // rows per work item of the band loop
    unsigned *status;
    unsigned long long *counter;
};

__device__ __forceinline__ bool finite4c(const float4 &v)
{
    const float big = 3.402823466e38f;
    return fabsf(v.x) <= big && fabsf(v.y) <= big && fabsf(v.z) <= big && fabsf(v.w) <= big;
}

// The per-step cluster barrier.  A CTA barrier first orders every thread's
// shared-memory reads and writes of the step (its own band, the halo rows it
// stored into its neighbours, the remote patch nodes its cones read) before
// one cluster-scope fence by one thread; the arrivals are then relaxed and the
// wait acquires.  A release arrival by each of the 1024 threads costs a memory
// barrier per warp instead of one per CTA.
__device__ __forceinline__ void cluster_step_sync()
{
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("fence.acq_rel.cluster;" ::: "memory");
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
}

// Bits of band rows b .. b + 31 from the per-row source bitmap (bit i: row b + i holds a source).
__device__ __forceinline__ unsigned band_row_bits(const unsigned *rows, int nrw, int b)
{
    const int w = b >> 5;
    const unsigned lo = rows[w], hi = w + 1 < nrw ? rows[w + 1] : 0u;
    return __funnelshift_r(lo, hi, b & 31);
}

template <bool MAP>
__global__ void __launch_bounds__(kClusterThreads, 1) cluster_kernel(const __grid_constant__ ClusterArgs A)
{
    extern __shared__ __align__(16) float smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int G = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const FieldDesc &f = A.f;
    const int nx = f.nx, ny = f.ny;
    const float alpha = f.alpha, beta = f.beta, dt = f.dt;
    const int Q = nx >> 2;                            // float4 groups per row
    const int band = A.band;
    const int y0 = min(rank * band, ny), y1 = min(y0 + band, ny);
    const int rows = y1 - y0;
    const int nrw = (band + 31) >> 5;                 // words of the per-row source bitmap
    const size_t bsz = (size_t)(band + 2) * nx;       // floats per buffer: halo, band, halo
    int *s_cell = reinterpret_cast<int *>(smem + 2 * bsz);   // this band's sources, in source order
    float *s_emit = reinterpret_cast<float *>(s_cell + kClusterMaxSources);
    unsigned *s_rows = reinterpret_cast<unsigned *>(s_emit + kClusterMaxSources);
    // the cones' noise of a step, drawn a step ahead by the field warps that have no
    // rows: [2 steps][2 components][CL cone lanes]
    const int CL = kClusterThreads - A.field_warps * 32;
    float *s_noise = reinterpret_cast<float *>(s_rows + nrw);
    __shared__ int s_nsrc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // rows y0 - 1 .. y1 of C^n into buffer 0 (a halo row beyond a wall is the
    // edge row itself); this band's sources and the rows that hold one
    // (cells outside the grid are reported by CTA 0)
    if (rows > 0) {
        const float4 *in4 = reinterpret_cast<const float4 *>(A.Cin);
        float4 *b4 = reinterpret_cast<float4 *>(smem);
        for (int q = tid; q < (rows + 2) * Q; q += kClusterThreads) {
            const int lr = q / Q, x4 = q - lr * Q;
            const int gy = min(max(y0 - 1 + lr, 0), ny - 1);
            b4[q] = __ldg(in4 + (size_t)gy * Q + x4);
        }
    }
    for (int w = tid; w < nrw; w += kClusterThreads) s_rows[w] = 0u;
    __syncthreads();
    if (tid == 0) {
        int m = 0;
        for (int k = 0; k < A.n_src; ++k) {
            const int c = __ldg(A.src_cell + k);
            if (c < 0 || c >= nx * ny) {
                if (rank == 0) flag_status(A.status, kStatusBounds);
                continue;
            }
            const int y = c / nx;
            if (y >= y0 && y < y1 && m < kClusterMaxSources) {
                s_cell[m] = c - y0 * nx;              // index inside the band
                s_emit[m] = __ldg(A.src_emit + k);
                s_rows[(y - y0) >> 5] |= 1u << ((y - y0) & 31);
                ++m;
            }
        }
        s_nsrc = m;
    }

    const int fw = A.field_warps;
    const bool field_warp = warp < fw;
    // the band loop's work items: column blocks of 32 groups x runs of A.rows rows
    const int ncb = (Q + 31) >> 5;
    const int R = A.rows;
    const int n_items = rows > 0 ? ncb * ((rows + R - 1) / R) : 0;
    // field warps left without rows draw the noise of the next step (at most two draws a
    // lane), which takes Philox and Box-Muller off the cones' dependent chain
    const int idle = fw - min(n_items, fw);          // the host set pre_noise only where CL <= 64 idle
    const bool pre_noise = A.pre_noise != 0 && idle > 0;
    const bool noise_warp = pre_noise && field_warp && warp >= fw - idle;
    auto draw_noise = [&](int step, int buf) {       // noise of step `step` into buffer buf
        for (int i = (warp - (fw - idle)) * 32 + lane; i < CL; i += idle * 32) {
            const int ai = i * G + rank;
            float xi[2] = {0.f, 0.f};
            if (ai < A.n_axons) cone_noise<2>(A.c.key0, A.c.key1, (uint32_t)ai, A.step0 + (uint32_t)step, xi);
            s_noise[(2 * buf) * CL + i] = xi[0];
            s_noise[(2 * buf + 1) * CL + i] = xi[1];
        }
    };
    if (noise_warp) draw_noise(0, 0);

    // cone a = i * G + rank belongs to this CTA's cone lane i: its state stays in registers
    const int a = ((warp - fw) * 32 + lane) * G + rank;
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
    // the neighbours' buffers, as distributed shared memory: the upper one's
    // bottom halo row (its band is full) and the lower one's top halo row
    const bool up_wall = y0 == 0, dn_wall = y1 >= ny;
    float4 *const up_h0 = reinterpret_cast<float4 *>(cl.map_shared_rank(smem, max(rank - 1, 0))) + (size_t)(band + 1) * Q;
    float4 *const up_h1 = reinterpret_cast<float4 *>(cl.map_shared_rank(smem + bsz, max(rank - 1, 0))) +
                          (size_t)(band + 1) * Q;
    float4 *const dn_h0 = reinterpret_cast<float4 *>(cl.map_shared_rank(smem, min(rank + 1, G - 1)));
    float4 *const dn_h1 = reinterpret_cast<float4 *>(cl.map_shared_rank(smem + bsz, min(rank + 1, G - 1)));
    cl.sync();                                        // every band and halo loaded, every bitmap built
    const int ns = s_nsrc;

    int cb = 0;                                       // buffer holding C^n
    for (int s = 0; s < A.nsteps; ++s) {
        const float *C = smem + cb * bsz;
        float *N = smem + (cb ^ 1) * bsz;
        if (field_warp) {
            const float4 *c4 = reinterpret_cast<const float4 *>(C);
            float4 *o4 = reinterpret_cast<float4 *>(N);
            float4 *const uh = cb ? up_h0 : up_h1, *const dh = cb ? dn_h0 : dn_h1;   // halos of buffer cb ^ 1
            for (int it = warp; it < n_items; it += fw) {   // warp-uniform
                const int cbk = it % ncb, b0 = (it / ncb) * R, b1 = min(b0 + R, rows);
                const int x4 = cbk * 32 + lane;       // this lane's group in the row
                const bool xin = x4 < Q;
                const bool need_l = lane == 0 && x4 > 0, need_r = lane == 31 && x4 + 1 < Q;
                const bool wall_l = x4 == 0, wall_r = x4 + 1 >= Q;
                // lanes past the right edge read the last group and drop their results;
                // local row b + 1 is band row b (rows 0 and rows + 1 are the halos)
                const float4 *col = c4 + (xin ? x4 : Q - 1);
                float4 vm = col[b0 * Q];
                float4 vc = col[(b0 + 1) * Q];
                unsigned bits = 0;
#pragma unroll 4
                for (int b = b0; b < b1; ++b) {
                    const float4 vp = col[(b + 2) * Q];
                    if (((b - b0) & 31) == 0) bits = band_row_bits(s_rows, nrw, b);
                    float l = __shfl_up_sync(kFullC, vc.w, 1);
                    float r = __shfl_down_sync(kFullC, vc.x, 1);
                    if (need_l) l = C[(size_t)(b + 1) * nx + 4 * x4 - 1];
                    if (need_r) r = C[(size_t)(b + 1) * nx + 4 * x4 + 4];
                    if (wall_l) l = vc.x;             // a wall: the missing neighbour is the node itself
                    if (wall_r) r = vc.w;
                    float4 o;
                    o.x = node_update2(vc.x, l, vc.y, vm.x, vp.x, alpha, beta);
                    o.y = node_update2(vc.y, vc.x, vc.z, vm.y, vp.y, alpha, beta);
                    o.z = node_update2(vc.z, vc.y, vc.w, vm.z, vp.z, alpha, beta);
                    o.w = node_update2(vc.w, vc.z, r, vm.w, vp.w, alpha, beta);
                    if constexpr (MAP) {
                        const float4 m = __ldg(reinterpret_cast<const float4 *>(A.map) + (size_t)(y0 + b) * Q +
                                               (xin ? x4 : 0));
                        o.x = fmaf(dt, m.x, o.x);
                        o.y = fmaf(dt, m.y, o.y);
                        o.z = fmaf(dt, m.z, o.z);
                        o.w = fmaf(dt, m.w, o.w);
                    }
                    if (bits & 1u) {                  // the row's sources at these nodes, in source order
                        const int c0 = b * nx + 4 * x4;
                        for (int k = 0; k < ns; ++k) {
                            const int rel = s_cell[k] - c0;
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
                    if (xin) {
                        o4[(size_t)(b + 1) * Q + x4] = o;
                        if (b == 0) {                 // the upper neighbour's bottom halo, or our own at a wall
                            if (up_wall) o4[x4] = o;
                            else uh[x4] = o;
                        }
                        if (b == rows - 1) {          // the lower neighbour's top halo, or our own at a wall
                            if (dn_wall) o4[(size_t)(rows + 1) * Q + x4] = o;
                            else dh[x4] = o;
                        }
                    }
                    vm = vc;
                    vc = vp;
                }
            }
            if (noise_warp && s + 1 < A.nsteps) draw_noise(s + 1, (s + 1) & 1);
        } else if (has_cone) {
            float xi[2];
            if (pre_noise) {
                const int i = (warp - fw) * 32 + lane;
                xi[0] = s_noise[(2 * (s & 1)) * CL + i];
                xi[1] = s_noise[(2 * (s & 1) + 1) * CL + i];
            } else {
                cone_noise<2>(A.c.key0, A.c.key1, (uint32_t)a, A.step0 + (uint32_t)s, xi);
            }
            if (act) {
                ++n_live;
                // every node from its owner's buffer through the cluster's shared-memory window
                // (this CTA's own too): no branch between the 12 loads, so they are issued
                // back to back
                auto ld = [&](int i, int j, int) {
                    const int owner = min(j / band, G - 1);
                    const float *b = cl.map_shared_rank(C, owner);
                    return b[(size_t)(j - owner * band + 1) * nx + i];
                };
                act = cone_step_rule<2>(f, A.c, ld, xi, p, d, A.src_xyz, A.n_src, stop ? A.n_src : 0);
                const float big = 3.402823466e38f;
                if (!(fabsf(p[0]) <= big && fabsf(p[1]) <= big && fabsf(d[0]) <= big && fabsf(d[1]) <= big))
                    bad = true;
            }
        }
        cluster_step_sync();                          // C^{n+1} and its halos complete everywhere; C^n no longer read
        cb ^= 1;
    }

    // buffer cb holds C^{n+k}, the other C^{n+k-1}: the band's rows to global memory;
    // non-finite values persist, so testing the last step's output covers the call
    if (rows > 0) {
        const float4 *c4 = reinterpret_cast<const float4 *>(smem + cb * bsz) + Q;
        const float4 *p4 = reinterpret_cast<const float4 *>(smem + (cb ^ 1) * bsz) + Q;
        float4 *out4 = reinterpret_cast<float4 *>(A.Cout) + (size_t)y0 * Q;
        float4 *prev4 = reinterpret_cast<float4 *>(A.Cprev) + (size_t)y0 * Q;
        for (int q = tid; q < rows * Q; q += kClusterThreads) {
            const float4 v = c4[q];
            bad |= !finite4c(v);
            out4[q] = v;
            prev4[q] = p4[q];
        }
    }
    if (has_cone) {
        A.pos[a] = p[0];
        A.pos[A.n_axons + a] = p[1];
        A.dir[a] = d[0];
        A.dir[A.n_axons + a] = d[1];
        A.active[a] = act ? 1 : 0;
    }
    if (__any_sync(kFullC, bad) && lane == 0) flag_status(A.status, kStatusNonFinite);
    if (!field_warp) {                                // warp-uniform
        const unsigned tot = __reduce_add_sync(kFullC, n_live);
        if (lane == 0 && tot) atomicAdd(A.counter, (unsigned long long)tot);
    }
    cl.sync();                                        // no CTA leaves while another may still read its memory
}

int cluster_band(const Sim &s, int G) { return (s.fd.ny + G - 1) / G; }

// The launch's split of a CTA's warps: field warps, and runs of rows just tall
// enough that every field warp has at most one work item; the cones' noise is
// drawn a step ahead when the fullest band leaves field warps without rows
// enough for at most two draws a lane.
struct ClusterSplit {
    int field_warps, rows, cone_lanes;
    bool pre_noise;
};

ClusterSplit cluster_split(const Sim &s, int G)
{
    ClusterSplit k;
    const int band = cluster_band(s, G);
    const int cones_per_cta = (s.n_axons + G - 1) / G;
    k.cone_lanes = (cones_per_cta + 31) / 32 * 32;
    k.field_warps = kClusterThreads / 32 - k.cone_lanes / 32;
    const int ncb = (s.fd.nx / 4 + 31) / 32;
    k.rows = std::max(1, (band * ncb + k.field_warps - 1) / k.field_warps);
    const int items = ncb * ((band + k.rows - 1) / k.rows);
    const int idle = k.field_warps - std::min(items, k.field_warps);
    k.pre_noise = k.cone_lanes > 0 && idle > 0 && k.cone_lanes <= 64 * idle;
    return k;
}

size_t cluster_smem_bytes(const Sim &s, int G)
{
    const int band = cluster_band(s, G);
    const ClusterSplit k = cluster_split(s, G);
    return 2 * sizeof(float) * (size_t)(band + 2) * s.fd.nx + 8 * (size_t)kClusterMaxSources +
           4 * (size_t)((band + 31) / 32) + (k.pre_noise ? 4 * sizeof(float) * (size_t)k.cone_lanes : 0);
}

// Dynamic shared memory a CTA may ask for: the per-block opt-in maximum less
// 1 KB for the kernel's static shared memory (the band's source count).
int cluster_smem_limit()
{
    static int limit = -1;
    if (limit < 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 0;
        limit = v > 1024 ? v - 1024 : 0;
    }
    return limit;
}

bool cluster_launch_ok()
{
    static int ok = -1;
    if (ok < 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        ok = cudaDeviceGetAttribute(&v, cudaDevAttrClusterLaunch, dev) == cudaSuccess && v ? 1 : 0;
    }
    return ok == 1;
}

// The kernels' function attributes (shared-memory allowance, non-portable
// cluster sizes) are per device: set them once on every device this process
// launches on.
bool cluster_attrs(bool map)
{
    static unsigned long long attr_set[2] = {0ull, 0ull};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (attr_set[map] & bit) return true;
    const void *fn = map ? (const void *)cluster_kernel<true> : (const void *)cluster_kernel<false>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, cluster_smem_limit()) != cudaSuccess)
        return false;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();                           // the portable size still works
    }
    attr_set[map] |= bit;
    return true;
}

cudaLaunchConfig_t cluster_config(int G, size_t smem, cudaStream_t stream, cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Whether a cluster of G CTAs takes this simulation: the shape rules, and the
// device able to schedule one such cluster (the occupancy query).
bool cluster_fits(const Sim &s, int G)
{
    if (s.fd.ny < 2 * G || s.n_axons > G * kClusterMaxConeWarps * 32) return false;
    const size_t smem = cluster_smem_bytes(s, G);
    if (smem > (size_t)cluster_smem_limit()) return false;
    const bool map = s.src_map != nullptr;
    if (!cluster_attrs(map)) return false;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(G, smem, nullptr, attr);
    int n = 0;
    const cudaError_t e = map ? cudaOccupancyMaxActiveClusters(&n, cluster_kernel<true>, &cfg)
                              : cudaOccupancyMaxActiveClusters(&n, cluster_kernel<false>, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n >= 1;
}

}  // namespace

int cluster_ctas(const Sim &s)
{
    if (s.cluster_pick >= 0) return s.cluster_pick;
    int G = 0;
    if (s.fd.dim == 2 && s.vec4 && s.n_src <= kClusterMaxSources && cluster_launch_ok()) {
        if (s.cluster_opt) G = cluster_fits(s, s.cluster_opt) ? s.cluster_opt : 0;
        else if (cluster_fits(s, kClusterSizeLarge)) G = kClusterSizeLarge;
        else if (cluster_fits(s, kClusterSize)) G = kClusterSize;
    }
    s.cluster_pick = G;                               // a cache: the answer depends only on fixed fields
    return G;
}

bool cluster_supported(const Sim &s) { return cluster_ctas(s) > 0; }

bool cluster_preferred(const Sim &s)
{
    const int G = cluster_ctas(s);
    if (!G) return false;
    const long long cells = (long long)s.fd.nx * s.fd.ny;
    return cells >= 4096 && (s.n_axons + G - 1) / G <= 128 && (long long)cluster_band(s, G) * s.fd.nx <= 16384;
}

int run_cluster_if_supported(Sim &s, int nsteps)
{
    if (s.path != CUE_PATH_AUTO && s.path != CUE_PATH_CLUSTER) return 1;
    const int G = cluster_ctas(s);
    if (!G) return s.path == CUE_PATH_CLUSTER ? CUE_ERR_ARG : 1;
    if (nsteps <= 0) return CUE_OK;
    if (s.cd.stop_r2 >= 0.0f && s.n_src > 0 && !s.src_xyz_ready) {
        if (launch_src_xyz(s) != cudaSuccess) return CUE_ERR_CUDA;
        s.src_xyz_ready = true;
    }
    const size_t smem = cluster_smem_bytes(s, G);
    const bool map = s.src_map != nullptr;
    if (!cluster_attrs(map)) return CUE_ERR_CUDA;
    ClusterArgs A{};
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
    A.band = cluster_band(s, G);
    const ClusterSplit split = cluster_split(s, G);
    A.field_warps = split.field_warps;
    A.rows = split.rows;
    A.pre_noise = split.pre_noise ? 1 : 0;
    A.status = s.status();
    A.counter = s.cone_counter();
    for (int done = 0; done < nsteps;) {              // launches of at most kPersistMaxSteps steps
        const int k = std::min(nsteps - done, kPersistMaxSteps);
        A.Cin = s.field[s.cur];
        A.Cout = s.field[s.cur ^ (k & 1)];
        A.Cprev = s.field[s.cur ^ (k & 1) ^ 1];
        A.nsteps = k;
        A.step0 = (uint32_t)s.cone_step;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_config(G, smem, s.stream, attr);
        timing_begin(s);
        cudaError_t e = map ? cudaLaunchKernelEx(&cfg, cluster_kernel<true>, A)
                            : cudaLaunchKernelEx(&cfg, cluster_kernel<false>, A);
        timing_end(s);
        s.launches++;
        if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return CUE_ERR_CUDA;
        s.cur ^= (k & 1);
        s.field_step += k;
        s.cone_step += k;
        done += k;
    }
    s.cluster_used = true;
    s.cluster_last = G;
    return CUE_OK;
}

}  // namespace cue
