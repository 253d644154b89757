// k_cluster.cu -- small 2D grids spread over a thread-block cluster for a
// whole call.
//
// One cluster of G CTAs (G = 8, one per SM) holds the field in distributed
// shared memory: CTA r owns a band of rows, kept in its shared memory in two
// buffers with one halo row above and below.  A step is: copy the two halo
// rows of the current buffer from the neighbouring CTAs' shared memory
// (distributed shared memory loads), update the band into the other buffer,
// step this CTA's cones on the current buffer (a cone's 12-node patch may lie
// in another CTA's band: those nodes are read from that CTA's shared memory),
// then one cluster barrier.  Global memory is read at the start (field,
// sources, cone state) and written at the end (both buffers, cone state).
// The single-SM resident kernel (k_resident.cu) issues every instruction of a
// step on one SM; here eight SMs share them and meet at a hardware cluster
// barrier, which has no software wait.
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
    int band;                    // rows per CTA (the last CTA may own fewer)
    unsigned *status;
    unsigned long long *counter;
};

__device__ __forceinline__ bool finite4c(const float4 &v)
{
    const float big = 3.402823466e38f;
    return fabsf(v.x) <= big && fabsf(v.y) <= big && fabsf(v.z) <= big && fabsf(v.w) <= big;
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
    const int y0 = rank * band, y1 = min(y0 + band, ny);
    const int rows = max(y1 - y0, 0);
    const int stride = band + 2;                      // rows per buffer: halo, band, halo
    float *buf[2] = {smem, smem + (size_t)stride * nx};
    int *s_cell = reinterpret_cast<int *>(smem + 2 * (size_t)stride * nx);   // this band's sources, in order
    float *s_emit = reinterpret_cast<float *>(s_cell + kClusterMaxSources);
    __shared__ int s_nsrc;
    const int tid = threadIdx.x, lane = tid & 31;

    // this band's rows of C^n, its sources (cells outside the grid are reported by CTA 0)
    {
        const float4 *in4 = reinterpret_cast<const float4 *>(A.Cin);
        float4 *b4 = reinterpret_cast<float4 *>(buf[0] + nx);
        for (int q = tid; q < rows * Q; q += kClusterThreads) b4[q] = __ldg(in4 + (size_t)y0 * Q + q);
        if (tid == 0) {
            int m = 0;
            for (int k = 0; k < A.n_src; ++k) {
                const int c = __ldg(A.src_cell + k);
                if (c < 0 || c >= nx * ny) {
                    if (rank == 0) flag_status(A.status, kStatusBounds);
                    continue;
                }
                if (c / nx >= y0 && c / nx < y1 && m < kClusterMaxSources) {
                    s_cell[m] = c - y0 * nx;      // index inside the band
                    s_emit[m] = __ldg(A.src_emit + k);
                    ++m;
                }
            }
            s_nsrc = m;
        }
    }
    // cone a belongs to CTA a % G, thread a / G: its state stays in registers
    const int a = tid * G + rank;
    const bool has_cone = a < A.n_axons;
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
    // the other CTAs' buffers, as distributed shared memory
    float *up_buf[2] = {cl.map_shared_rank(buf[0], max(rank - 1, 0)), cl.map_shared_rank(buf[1], max(rank - 1, 0))};
    float *dn_buf[2] = {cl.map_shared_rank(buf[0], min(rank + 1, G - 1)),
                        cl.map_shared_rank(buf[1], min(rank + 1, G - 1))};
    cl.sync();                                        // every band loaded before anyone reads a neighbour's
    int cur = 0;
    for (int s = 0; s < A.nsteps; ++s) {
        float *C = buf[cur], *N = buf[cur ^ 1];
        // halo rows: the neighbours' edge rows of C^n (a wall: the band's own edge row)
        for (int x = tid; x < nx; x += kClusterThreads) {
            C[x] = y0 > 0 ? up_buf[cur][(size_t)band * nx + x] : C[nx + x];
            C[(size_t)(rows + 1) * nx + x] = y1 < ny ? dn_buf[cur][nx + x] : C[(size_t)rows * nx + x];
        }
        __syncthreads();
        // the band: groups of four nodes, the x neighbours read at the group's edges
        const int ns = s_nsrc;
        for (int q = tid; q < rows * Q; q += kClusterThreads) {
            const int r = q / Q, x4 = q - r * Q;
            const float *row = C + (size_t)(r + 1) * nx;
            const float4 vc = reinterpret_cast<const float4 *>(row)[x4];
            const float4 vm = reinterpret_cast<const float4 *>(row - nx)[x4];
            const float4 vp = reinterpret_cast<const float4 *>(row + nx)[x4];
            const float l = x4 > 0 ? row[4 * x4 - 1] : vc.x;          // a wall: the node itself
            const float rr = x4 + 1 < Q ? row[4 * x4 + 4] : vc.w;
            float4 o;
            o.x = node_update2(vc.x, l, vc.y, vm.x, vp.x, alpha, beta);
            o.y = node_update2(vc.y, vc.x, vc.z, vm.y, vp.y, alpha, beta);
            o.z = node_update2(vc.z, vc.y, vc.w, vm.z, vp.z, alpha, beta);
            o.w = node_update2(vc.w, vc.z, rr, vm.w, vp.w, alpha, beta);
            if constexpr (MAP) {
                const float4 m = __ldg(reinterpret_cast<const float4 *>(A.map) + (size_t)y0 * Q + q);
                o.x = fmaf(dt, m.x, o.x);
                o.y = fmaf(dt, m.y, o.y);
                o.z = fmaf(dt, m.z, o.z);
                o.w = fmaf(dt, m.w, o.w);
            }
            for (int k = 0; k < ns; ++k) {            // the band's sources at these nodes, in source order
                const int rel = s_cell[k] - 4 * q;
                if (rel >= 0 && rel < 4) {
                    const float em = s_emit[k];
                    if (rel == 0) o.x += em;
                    else if (rel == 1) o.y += em;
                    else if (rel == 2) o.z += em;
                    else o.w += em;
                }
            }
            reinterpret_cast<float4 *>(N + (size_t)(r + 1) * nx)[x4] = o;
        }
        // this CTA's cones on C^n: nodes of other bands from their CTAs' shared memory
        if (has_cone) {
            float xi[2];
            cone_noise<2>(A.c.key0, A.c.key1, (uint32_t)a, A.step0 + (uint32_t)s, xi);
            if (act) {
                ++n_live;
                auto ld = [&](int i, int j, int) {
                    const int owner = min(j / band, G - 1);
                    const float *b = owner == rank ? C : cl.map_shared_rank(C, owner);
                    return b[(size_t)(j - owner * band + 1) * nx + i];
                };
                act = cone_step_rule<2>(f, A.c, ld, xi, p, d, A.src_xyz, A.n_src, stop ? A.n_src : 0);
                const float big = 3.402823466e38f;
                if (!(fabsf(p[0]) <= big && fabsf(p[1]) <= big && fabsf(d[0]) <= big && fabsf(d[1]) <= big))
                    bad = true;
            }
        }
        cl.sync();                                    // C^{n+1} complete everywhere; C^n no longer read
        cur ^= 1;
    }

    // buf[cur] holds C^{n+k}, the other C^{n+k-1}: the band's rows to global memory
    {
        const float4 *c4 = reinterpret_cast<const float4 *>(buf[cur] + nx);
        const float4 *p4 = reinterpret_cast<const float4 *>(buf[cur ^ 1] + nx);
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
    const unsigned tot = __reduce_add_sync(kFullC, n_live);
    if (lane == 0 && tot) atomicAdd(A.counter, (unsigned long long)tot);
    cl.sync();                                        // no CTA leaves while another may still read its memory
}

int cluster_band(const Sim &s) { return (s.fd.ny + kClusterSize - 1) / kClusterSize; }

size_t cluster_smem_bytes(const Sim &s)
{
    return 2 * sizeof(float) * (size_t)(cluster_band(s) + 2) * s.fd.nx + 8 * (size_t)kClusterMaxSources;
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

}  // namespace

bool cluster_supported(const Sim &s)
{
    return s.fd.dim == 2 && s.vec4 && s.fd.ny >= 2 * kClusterSize && s.n_axons <= kClusterSize * kClusterThreads &&
           s.n_src <= kClusterMaxSources && cluster_launch_ok() &&
           cluster_smem_bytes(s) <= (size_t)cluster_smem_limit();
}

int run_cluster_if_supported(Sim &s, int nsteps)
{
    if (s.path != CUE_PATH_AUTO && s.path != CUE_PATH_CLUSTER) return 1;
    if (!cluster_supported(s)) return s.path == CUE_PATH_CLUSTER ? CUE_ERR_ARG : 1;
    if (nsteps <= 0) return CUE_OK;
    if (s.cd.stop_r2 >= 0.0f && s.n_src > 0 && !s.src_xyz_ready) {
        if (launch_src_xyz(s) != cudaSuccess) return CUE_ERR_CUDA;
        s.src_xyz_ready = true;
    }
    const size_t smem = cluster_smem_bytes(s);
    const bool map = s.src_map != nullptr;
    // the shared-memory allowance is a per-device function attribute: set it once per device
    static unsigned long long attr_set[2] = {0ull, 0ull};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CUE_ERR_CUDA;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!(attr_set[map] & bit)) {
        cudaError_t e = map ? cudaFuncSetAttribute(cluster_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   cluster_smem_limit())
                            : cudaFuncSetAttribute(cluster_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   cluster_smem_limit());
        if (e != cudaSuccess) return CUE_ERR_CUDA;
        attr_set[map] |= bit;
    }
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
    A.band = cluster_band(s);
    A.status = s.status();
    A.counter = s.cone_counter();
    for (int done = 0; done < nsteps;) {              // launches of at most kPersistMaxSteps steps
        const int k = std::min(nsteps - done, kPersistMaxSteps);
        A.Cin = s.field[s.cur];
        A.Cout = s.field[s.cur ^ (k & 1)];
        A.Cprev = s.field[s.cur ^ (k & 1) ^ 1];
        A.nsteps = k;
        A.step0 = (uint32_t)s.cone_step;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kClusterSize);
        cfg.blockDim = dim3(kClusterThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s.stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kClusterSize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
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
    return CUE_OK;
}

}  // namespace cue
