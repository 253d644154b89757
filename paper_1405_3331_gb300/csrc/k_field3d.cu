// k_field3d.cu -- the 3D field step (rows a1, a2, a7) as a TMA-pipelined
// 2.5D stencil: each CTA owns an x-y column tile (128 x 16 nodes) and marches
// along z through a chunk of planes.  One thread issues TMA tensor copies of
// whole planes (tile plus a one-node halo in y and a four-node halo in x, for
// 16-byte TMA coordinates) into a ring of four shared-memory stages, keeping
// two planes ahead of the one being computed; every thread computes four
// nodes per plane from shared memory (x neighbours by warp shuffle) and
// writes them with one 16-byte store.  HBM traffic: one read and one write
// per node (8 B per node update) plus the halo overlap.  A ninth warp per CTA
// steps the CTA's share of the growth cones on the input field meanwhile (its
// gathers are dependent global loads; the eight field warps synchronise among
// themselves on a named barrier and never wait for it), and after the last
// plane the field warps add the point sources of the CTA's box.
//
// Update (Sec. 5.2, Sec. 4.3): C' = beta C + alpha * (sum of the six axis
// neighbours) [+ dt M], a neighbour missing at a wall replaced by the node
// itself (node_update3, the same expression as the other field kernels).
#include <cuda.h>

#include "cue_internal.h"

namespace cue {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTX = 128;              // interior columns per tile (32 lanes x float4)
constexpr int kHX = 4;                // x halo (TMA coordinates must be 16-byte aligned)
constexpr int kBoxX = kTX + 2 * kHX;  // 136 floats = 544 bytes per row
constexpr int kBY = 16;               // interior rows per tile
constexpr int kBoxY = kBY + 2;
constexpr int kStages = 4;
constexpr int kAhead = kStages - 2;   // planes in flight beyond the three being read
constexpr int kThreads3 = 256;        // field warps: 8 warps x 2 rows
constexpr int kLaunch3 = kThreads3 + 32;  // + one warp for the block's cones
constexpr int kStageFloats = kBoxX * kBoxY;                   // one plane tile (9,792 bytes)
// TMA writes to shared memory must start on a 128-byte boundary: stages are
// spaced by the plane size rounded up to 128 bytes.
constexpr int kStageStride = ((kStageFloats * 4 + 127) / 128) * 128 / 4;
static_assert((kStageStride * 4) % 128 == 0, "TMA stage stride must be a multiple of 128 bytes");
constexpr long long kWaitLimit = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase)
{
    for (long long i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

struct Field3Args {
    FieldDesc f;
    float *Cout;
    const float *M;      // dense rate map or null
    int ntx, nty, zchunk;
    unsigned *status;
    // the same step's cones (they read the input buffer, which no block of this
    // launch writes): the cone warp of block b steps cones [b cone_per,
    // (b+1) cone_per), 32 at a time; cone_per 0 = none
    int cone_per;
    ConeDesc c;
    uint32_t step;
    int n;
    const float *Cin;
    float *pos, *dir;
    uint8_t *active;
    const float *src_xyz;
    int n_stop;          // sources of the stop test (0: off)
    unsigned long long *counter;
    // point sources, added by the field block that owns their node (n_add 0: none)
    const int32_t *src_cell;
    const float *src_emit;
    int n_add;
};

// Cone a (inr: a is one of this block's cones): the plain cone kernel's step
// (same functions, same order), with the source coordinates of the stop test
// read from global memory.  Called by whole warps (the active count is a
// warp vote).
__device__ __forceinline__ void cone_one3(const Field3Args &A, int a, bool inr)
{
    const FieldDesc &f = A.f;
    const int n = A.n;
    const uint8_t act = inr ? A.active[a] : 0;
    float p[3], d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        p[i] = inr ? A.pos[(size_t)i * n + a] : 0.0f;
        d[i] = inr ? A.dir[(size_t)i * n + a] : 0.0f;
    }
    float xi[3];
    cone_noise<3>(A.c.key0, A.c.key1, (uint32_t)a, A.step, xi);
    const bool live = inr && act;
    count_active(A.counter, live);
    if (!live) return;
    const size_t sy = f.nx, sz = (size_t)f.nx * f.ny;
    auto ld = [&](int i, int j, int k) { return __ldg(A.Cin + (size_t)i + sy * j + sz * k); };
    const bool alive = cone_step_rule<3>(f, A.c, ld, xi, p, d, A.src_xyz, A.n_stop, A.n_stop);
    bool bad = false;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        A.pos[(size_t)i * n + a] = p[i];
        A.dir[(size_t)i * n + a] = d[i];
        bad |= !(fabsf(p[i]) <= 3.402823466e38f) || !(fabsf(d[i]) <= 3.402823466e38f);
    }
    if (!alive) A.active[a] = 0;
    if (bad) flag_status(A.status, kStatusNonFinite);
}

// The field warps meet at named barrier 1 (kThreads3 threads), so the cone
// warp never holds them up.
__device__ __forceinline__ void field_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kThreads3) : "memory"); }

__device__ __forceinline__ bool field_sync_or(bool p)
{
    unsigned r;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, 1, %2, pi;\n"
        " selp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"((unsigned)p), "n"(kThreads3)
        : "memory");
    return r != 0;
}

// CONES: the launch carries the cone warp (kLaunch3 threads); otherwise the
// field warps alone, with the register budget of 256 threads.
template <bool MAP, bool CONES>
__global__ void __launch_bounds__(CONES ? kLaunch3 : kThreads3, 4)
    field3d_tma_kernel(const __grid_constant__ CUtensorMap tmap, const Field3Args A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);                 // kStages barriers
    float *stage = reinterpret_cast<float *>(smem_raw + 128);                // kStages x kStageStride
    const FieldDesc &f = A.f;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int b = blockIdx.x;
    const int fb = b;                            // field block index
    const int tx = b % A.ntx;
    b /= A.ntx;
    const int ty = b % A.nty;
    const int zc = b / A.nty;
    const int x0 = tx * kTX, y0 = ty * kBY;
    const int zs = zc * A.zchunk, ze = min(zs + A.zchunk, f.nz);
    const int plo = max(zs - 1, 0), phi = min(ze, f.nz - 1);   // planes this CTA reads
    const unsigned bytes = kStageFloats * sizeof(float);

    // a programmatic dependent launch: the next step's CTAs may be scheduled as this
    // launch's CTAs finish; this one's set-up overlaps the previous launch's tail, and
    // griddepcontrol.wait (a no-op without the launch attribute) returns once the
    // previous launch has completed and its writes (the field, the cones) are visible
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    auto issue = [&](int p) {      // plane p into stage (p - plo) % kStages
        const int s = (p - plo) % kStages;
        mbar_expect_tx(&bar[s], bytes);
        tma_load_3d(stage + s * kStageStride, &tmap, &bar[s], x0 - kHX, y0 - 1, p);
    };
    auto wait = [&](int p) {
        const int k = p - plo;
        return mbar_wait_bounded(&bar[k % kStages], (unsigned)((k / kStages) & 1));
    };
    if (CONES && warp == kThreads3 / 32) {        // the cone warp: this block's cones, alongside the field
        if (A.cone_per > 0) {
            const int first = fb * A.cone_per;
            const int cnt = min(A.cone_per, A.n - first);
            for (int base = 0; base < cnt; base += 32)  // whole warp each round (the active count is a vote)
                cone_one3(A, first + base + lane, base + lane < cnt);
        }
        return;
    }
    if (tid == 0)
        for (int p = plo; p <= min(phi, plo + kStages - 2); ++p) issue(p);

    const int gx = x0 + 4 * lane;
    const bool xin = gx < f.nx;
    const bool wl = gx == 0, wr = gx + 3 == f.nx - 1;
    const float2 alpha2 = make_float2(f.alpha, f.alpha), beta2 = make_float2(f.beta, f.beta);
    const float4 *s4 = reinterpret_cast<const float4 *>(stage);
    bool tmo = false, bad = false;
    for (int p = plo; p <= zs; ++p)          // planes z-1 (if any) and z of the first step
        if (!wait(p)) tmo = true;
    for (int z = zs; z < ze; ++z) {
        // keep kAhead planes ahead: plane z+kAhead into the stage plane z-2 used
        if (tid == 0 && z + kAhead <= phi && z + kAhead >= plo + kStages - 1) issue(z + kAhead);
        if (z + 1 <= phi && !wait(z + 1)) tmo = true;
        if (field_sync_or(tmo)) {
            if (tid == 0) {
                flag_status(A.status, kStatusTimeout);
                for (int p = plo; p <= phi; ++p) wait(p);    // let in-flight copies land (bounded)
            }
            return;
        }
        const int sc = (z - plo) % kStages;
        const int sm = z > 0 ? (z - 1 - plo) % kStages : sc;           // z wall: the plane itself
        const int sp = z + 1 < f.nz ? (z + 1 - plo) % kStages : sc;
        const float *Pc = stage + sc * kStageStride;
#pragma unroll
        for (int rr = 0; rr < kBY / 8; ++rr) {
            const int r = warp * (kBY / 8) + rr;          // interior row 0..15 -> tile row r + 1
            const int gy = y0 + r;
            const int row = (r + 1) * kBoxX;
            const int col4 = (kHX + 4 * lane) / 4;
            const float4 c = s4[(sc * kStageStride + row) / 4 + col4];
            float4 ym = s4[(sc * kStageStride + row - kBoxX) / 4 + col4];
            float4 yp = s4[(sc * kStageStride + row + kBoxX) / 4 + col4];
            const float4 zm = s4[(sm * kStageStride + row) / 4 + col4];
            const float4 zp = s4[(sp * kStageStride + row) / 4 + col4];
            if (gy == 0) ym = c;
            if (gy == f.ny - 1) yp = c;
            float l = __shfl_up_sync(kFull, c.w, 1);
            float rt = __shfl_down_sync(kFull, c.x, 1);
            if (lane == 0) l = Pc[row + kHX - 1];
            if (lane == 31) rt = Pc[row + kHX + kTX];
            if (wl) l = c.x;
            if (wr) rt = c.w;
            if (xin && gy < f.ny) {
                float4 o = node_update3_x4(c, l, rt, ym, yp, zm, zp, alpha2, beta2);
                const size_t idx = ((size_t)z * f.ny + gy) * f.nx + gx;
                if constexpr (MAP) {
                    const float4 m = __ldg(reinterpret_cast<const float4 *>(A.M + idx));
                    o.x = fmaf(f.dt, m.x, o.x);
                    o.y = fmaf(f.dt, m.y, o.y);
                    o.z = fmaf(f.dt, m.z, o.z);
                    o.w = fmaf(f.dt, m.w, o.w);
                }
                bad |= !(fabsf(o.x) <= 3.4e38f && fabsf(o.y) <= 3.4e38f && fabsf(o.z) <= 3.4e38f &&
                         fabsf(o.w) <= 3.4e38f);
                *reinterpret_cast<float4 *>(A.Cout + idx) = o;
            }
        }
        field_sync();          // every field thread is done with plane z-1's stage before it is refilled
    }
    if (__any_sync(kFull, bad) && lane == 0) flag_status(A.status, kStatusNonFinite);
    // point sources in this block's box, after its stores (the last barrier above)
    if (A.n_add > 0) {
        const long long n_cells = (long long)f.nx * f.ny * f.nz;
        for (int k = tid; k < A.n_add; k += kThreads3) {
            const long long c = A.src_cell[k];
            if (c < 0 || c >= n_cells) {
                if (fb == 0) flag_status(A.status, kStatusBounds);
                continue;
            }
            const int cx = (int)(c % f.nx), cy = (int)((c / f.nx) % f.ny), cz = (int)(c / ((long long)f.nx * f.ny));
            if (cx >= x0 && cx < x0 + kTX && cy >= y0 && cy < y0 + kBY && cz >= zs && cz < ze)
                atomicAdd(A.Cout + c, A.src_emit[k]);
        }
    }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn3()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

int sm_count3()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 152;
}

}  // namespace

// Tensor maps of the two field buffers as TMA sources; false if unavailable.
bool field3d_tma_prepare(Sim &s)
{
    if (s.tmap3_ready) return true;
    if (s.fd.dim != 3 || !s.vec4) return false;
    EncodeTiledFn fn = encode_fn3();
    if (!fn) return false;
    for (int b = 0; b < 2; ++b) {
        cuuint64_t dims[3] = {(cuuint64_t)s.fd.nx, (cuuint64_t)s.fd.ny, (cuuint64_t)s.fd.nz};
        cuuint64_t strides[2] = {(cuuint64_t)s.fd.nx * sizeof(float), (cuuint64_t)s.fd.nx * s.fd.ny * sizeof(float)};
        cuuint32_t box[3] = {(cuuint32_t)kBoxX, (cuuint32_t)kBoxY, 1};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = fn(reinterpret_cast<CUtensorMap *>(s.tmap3[b]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, s.field[b],
                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    const int smem = 128 + kStages * kStageStride * (int)sizeof(float);
    if (cudaFuncSetAttribute(field3d_tma_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(field3d_tma_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(field3d_tma_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(field3d_tma_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess)
        return false;
    s.tmap3_ready = true;
    return true;
}

cudaError_t launch_field3d_tma(Sim &s, int in_buffer, float *Cout, bool *cones_done, bool *sources_done)
{
    Field3Args A{};
    A.f = s.fd;
    A.c = s.cd;
    A.step = (uint32_t)s.cone_step;
    A.n = s.n_axons;
    A.Cin = s.field[in_buffer];
    A.pos = s.pos;
    A.dir = s.dir;
    A.active = s.active;
    A.src_xyz = s.src_xyz();
    A.n_stop = (s.cd.stop_r2 >= 0.0f && s.n_src > 0) ? s.n_src : 0;
    A.counter = s.cone_counter();
    A.src_cell = s.src_cell;
    A.src_emit = s.src_emit;
    // each field block scans the whole source list, so only short lists are merged
    A.n_add = (sources_done && s.n_src <= kTma3BlockSources) ? s.n_src : 0;
    if (sources_done) *sources_done = A.n_add == s.n_src;
    A.Cout = Cout;
    A.M = s.src_map;
    A.ntx = (s.fd.nx + kTX - 1) / kTX;
    A.nty = (s.fd.ny + kBY - 1) / kBY;
    A.status = s.status();
    // at most one wave (four CTAs per SM resident): a CTA left for a second wave would
    // stream its whole chunk after the others; each CTA marches a chunk of z planes
    const long long cols = (long long)A.ntx * A.nty;
    long long chunks = 4LL * sm_count3() / cols;
    if (chunks < 1) chunks = 1;
    if (chunks > s.fd.nz) chunks = s.fd.nz;
    A.zchunk = (int)((s.fd.nz + chunks - 1) / chunks);
    chunks = (s.fd.nz + A.zchunk - 1) / A.zchunk;
    const unsigned grid = (unsigned)(cols * chunks);
    // the cones ride along (at most 8 rounds of the cone warp per block)
    const long long per = ((long long)s.n_axons + grid - 1) / grid;
    A.cone_per = (cones_done && s.n_axons > 0 && per <= kThreads3) ? (int)per : 0;
    if (cones_done) *cones_done = A.cone_per > 0 || s.n_axons == 0;
    const int smem = 128 + kStages * kStageStride * (int)sizeof(float);
    const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(s.tmap3[in_buffer]);
    const bool cones = A.cone_per > 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(cones ? kLaunch3 : kThreads3);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (s.src_map)
        e = cones ? cudaLaunchKernelEx(&cfg, field3d_tma_kernel<true, true>, *map, A)
                  : cudaLaunchKernelEx(&cfg, field3d_tma_kernel<true, false>, *map, A);
    else
        e = cones ? cudaLaunchKernelEx(&cfg, field3d_tma_kernel<false, true>, *map, A)
                  : cudaLaunchKernelEx(&cfg, field3d_tma_kernel<false, false>, *map, A);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace cue
