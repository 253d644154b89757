// k_fused3d.cu -- the temporally blocked 3D path: one launch advances the
// field AND the growth cones two steps (rows a1-a7), so the field makes one
// HBM read per two steps instead of one per step.
//
// Geometry.  The grid is cut into boxes: a column tile of 128 x TY nodes in
// x-y times a chunk of ZC planes in z; one CTA per box, two resident per SM,
// and the host picks TY and the chunk count for the fewest waves of the
// least work (256^3: TY = 14, eight chunks of 32 planes, 304 boxes).  Each
// CTA marches its box along z:
//   level 0 (C^n)      input planes arrive by TMA tensor copies (the box's
//                      136 x (TY + 8) nodes: a 4-node halo in x, for 16-byte
//                      TMA coordinates, and 4 in y) into a ring of kR0 stages,
//                      kD planes ahead of the one consumed; planes further
//                      ahead are prefetched into L2 by the tensor prefetch;
//   level 1 (C^{n+1})  plane p - 1 is computed from input planes p - 2 .. p
//                      while plane p lands, over the halo shrunk by one node
//                      (box rows 2 .. TY + 6), into a ring of kR1 planes and
//                      out to a scratch copy of the field in the workspace;
//   level 2 (C^{n+2})  plane p - 2 of the interior is computed from level-1
//                      planes p - 3 .. p - 1 and stored to the output buffer.
// Each field thread owns up to kItems float4 groups of level-1 nodes for the
// whole march and keeps its own nodes of the last planes in registers (input
// plane i - 1, level-1 planes i - 3 and i - 2), so a level reads little else
// than the y neighbours from shared memory (x neighbours by warp shuffle).  The halo H = 4 (y, and the z planes zs - 3 .. ze + 3) is
// K + 1 + ceil((K - 1) step_len / h) for K = 2 and step_len <= h: the field
// of the interior needs K, the cones add their drift and their 4-node
// footprint.
//
// Cones.  Each box's cones (binned by position as the previous launch's cones
// finished) are stepped by two cone warps that never hold up the field warps.
// Sub-step 0 reads C^n from the input buffer, sub-step 1 reads C^{n+1} from
// the scratch copy; a level-1 plane is published there (an acquire/release
// progress counter in shared memory) once the field warps have stored it,
// and a box writes every level-1 node its cones can reach (neighbouring boxes
// write the same values on their overlap).  The cone warps take the cones
// whose footprint planes have been published, in rounds of a whole warp, as
// the march passes them, so their gathers find the planes in L2 (just loaded
// by TMA, or just written).  A cone's last sub-step writes its state back and
// bins it for the next launch.
//
// Arithmetic: the same node update (node_update3), rate-map term and point
// sources in the same order as every other 3D kernel, and the same cone step
// (cone_step_rule<3>) on the same values, so the path equals the one-launch-
// per-step path bit for bit.
//
// Model: cue field on an Eulerian grid (Sec. 5.2) with sources of their own
// rates (Sec. 4.3); cone steering by vector addition (Sec. 3.5, Eq. 6-7) with
// stateless counter-based noise (Sec. 5.1) and Box-Muller (Sec. 3.2); stop
// tests on the bounds (Sec. 3.4) and squared source distance (Sec. 3.3).
#include <cuda.h>

#include <cmath>

#include "cue_internal.h"

namespace cue {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTX = 128;               // interior columns of a box
constexpr int kHX = 4;                 // x halo
constexpr int kW = kTX + 2 * kHX;      // 136 loaded columns
constexpr int kW4 = kW / 4;            // 34 float4 groups per row
constexpr int kH = 4;                  // y halo (rows) and the z reach of the march
constexpr int kFW = 8;                 // field warps
constexpr int kCW = 2;                 // cone warps
constexpr int kFT = 32 * kFW;
constexpr int kAllT = kFT + 32 * kCW;
constexpr int kItems = 3;              // level-1 groups per field thread: 34 (TY + 5) <= 3 * 256
constexpr int kD = 2;                  // input planes in flight (TMA into shared memory) ahead of the one consumed
constexpr int kPF = 6;                 // input planes prefetched into L2 this far ahead
constexpr int kR0 = kD + 3;            // input-plane ring: planes i - 2 .. i read, kD in flight
constexpr int kR1 = 3;                 // level-1 ring: plane i - 2 read, i - 1 written, one spare
constexpr int kConeCap = 512;          // cones of a box held in shared memory
constexpr int kMaxSrcF3 = 512;         // point sources in total on this path
constexpr int kMinTY = 8, kMaxTY = 16;
constexpr int kSmsGB300 = 152;         // SMs the geometry is chosen for
constexpr int kCtasPerSm = 2;
// dynamic shared memory a CTA may take with two resident per SM (228 KB per SM,
// 1 KB reserved per CTA, some bytes of static shared memory)
constexpr size_t kSmemPerCta = 233472 / kCtasPerSm - 1024 - 256;
constexpr long long kSpinLimit = 1LL << 24;  // cone-warp polls of the march's progress (~256 ns apart)
constexpr int kScanStep = 3;                 // planes the march advances between two cone scans
static_assert(kW4 * (kMaxTY + 5) <= kItems * kFT, "level-1 groups must fit the field threads");

constexpr int kBarField = 1;           // named barrier of the field warps

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool field_sync_or(bool p)
{
    unsigned r;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, %2, %3, pi;\n"
        " selp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"((unsigned)p), "n"(kBarField), "n"(kFT)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}

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

// As mbar_try_wait, but the thread may sleep in hardware up to `ns` nanoseconds
// (woken when the phase completes) instead of returning at once.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, unsigned phase, unsigned ns)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase), "r"(ns)
        : "memory");
    return ok != 0;
}

// Bounded wait (about a second at most): polls that sleep until the phase
// completes, so a waiting warp takes no issue slots from the others.
constexpr long long kSleepPolls = 1LL << 20;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase)
{
    for (long long i = 0; i < kSleepPolls; ++i)
        if (mbar_try_wait_sleep(bar, phase, 1000u)) return true;
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

// The same box of plane z into L2 only (no shared memory, no completion).
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *map, int x, int y, int z)
{
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}

// Wait for an input plane: one lane of the warp polls (bounded), then every lane
// observes the completed phase itself (which returns at once).
__device__ __forceinline__ bool warp_wait_plane(uint64_t *bar, unsigned phase, int lane)
{
    bool ok = true;
    if (lane == 0) ok = mbar_wait_bounded(bar, phase);
    ok = __shfl_sync(kFull, ok, 0);
    if (ok) mbar_try_wait(bar, phase);
    return ok;
}

__device__ __forceinline__ void add_comp(float4 &v, int k, float e)
{
    if (k == 0) v.x += e;
    else if (k == 1) v.y += e;
    else if (k == 2) v.z += e;
    else v.w += e;
}

__device__ __forceinline__ bool finite4(const float4 &v)
{
    return fabsf(v.x) <= 3.4e38f && fabsf(v.y) <= 3.4e38f && fabsf(v.z) <= 3.4e38f && fabsf(v.w) <= 3.4e38f;
}

struct F3Args {
    FieldDesc f;
    ConeDesc c;
    int TY, ntx, nty, ZC;
    int p0s, p1s;                 // floats per ring slot (input plane, level-1 plane)
    const float *Cin;             // C^n (the input buffer; the TMA source too)
    float *inter;                 // scratch copy of C^{n+1} (the level-1 nodes each box's cones can reach)
    float *Cout;                  // C^{n+2}
    const float *M;               // dense rate map or null
    uint32_t step0;
    int n;                        // cones
    float *pos, *dir;
    uint8_t *active;
    int *cnt_cur;                 // this launch's bin counts (each box clears its own once read)
    const int *bins_cur;
    int *cnt_next;                // the next launch's bins, filled as cones finish
    int *bins_next;
    int bin_cap;
    int *sched;                   // schedule words of the cones past kConeCap, by cone id
    const int32_t *src_cell;
    const float *src_emit;
    int n_src;
    const float *src_xyz;
    int n_stop;
    unsigned *status;
    unsigned long long *counter;
};

// Box of a position: the cell of each coordinate, clamped into the grid.
__device__ __forceinline__ int box_of3(const F3Args &A, const float *p)
{
    const FieldDesc &f = A.f;
    const int ix = clampi((int)floorf(p[0] * f.inv_h), 0, f.nx - 1);
    const int iy = clampi((int)floorf(p[1] * f.inv_h), 0, f.ny - 1);
    const int iz = clampi((int)floorf(p[2] * f.inv_h), 0, f.nz - 1);
    return ((iz / A.ZC) * A.nty + iy / A.TY) * A.ntx + ix / kTX;
}

// Newest plane of the footprint of a cone at height pz (the cell's lower
// corner clamped to nz - 2, as cell_of does, plus two).
__device__ __forceinline__ int need_of(const FieldDesc &f, float pz)
{
    const int lo = clampi((int)floorf(pz * f.inv_h), 0, f.nz - 2);
    return min(lo + 2, f.nz - 1);
}

// A cone's schedule word: the sub-step j it takes next and the newest plane its
// footprint reads (-1: done for this launch).
constexpr int kSchedDone = -1;
__device__ __forceinline__ int sched_word(int need, int j) { return need | (j << 24); }
// Ready at march progress `prog` (level-1 planes <= prog published; input planes
// <= prog + 1 loaded, so a sub-step-0 footprint is in L2 by then).
__device__ __forceinline__ bool sched_ready(int w, int prog)
{
    return w >= 0 && (w & 0xFFFFFF) <= prog + ((w >> 24) == 0 ? 1 : 0);
}

template <bool MAP, bool CONES>
__global__ void __launch_bounds__(CONES ? kAllT : kFT, kCtasPerSm)
    fused3d_kernel(const __grid_constant__ CUtensorMap tmap, const F3Args A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const FieldDesc &f = A.f;
    const int TY = A.TY;
    const int R = TY + 2 * kH;          // loaded rows
    const int L1R = TY + 5;             // level-1 rows (box rows 2 .. TY + 6)
    const int nL1 = kW4 * L1R;

    int b = blockIdx.x;
    const int box = b;
    const int tx = b % A.ntx;
    b /= A.ntx;
    const int ty = b % A.nty;
    const int ch = b / A.nty;
    const int ox = tx * kTX - kHX, oy = ty * TY - kH;          // global x, y of box node (0, 0)
    const int zs = ch * A.ZC, ze = min(zs + A.ZC, f.nz);
    const int ib = max(zs - 3, 0);                             // first input plane
    const int ilast = min(ze + 3, f.nz - 1);                   // last input plane
    const int l1_lo = max(zs - 2, 0), l1_hi = min(ze + 2, f.nz - 1);
    // last iteration: level-1 plane l1_hi is made at l1_hi + 1, level-2 plane ze - 1 at ze + 1
    const int iend = max(l1_hi + 1, ze + 1);
    const int npl = l1_hi - l1_lo + 1;

    // shared memory: barriers | input ring | level-1 ring | cones | sources
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    float *P0 = reinterpret_cast<float *>(smem_raw + 128);
    float *P1 = P0 + kR0 * A.p0s;
    float *cst = P1 + kR1 * A.p1s;                             // [6][kConeCap] px py pz dx dy dz
    int *cid = reinterpret_cast<int *>(cst + 6 * kConeCap);
    int *csch = cid + kConeCap;                                // schedule words
    int *dlist = csch + kConeCap;                              // per cone warp: kConeCap / kCW
    int *s_key = dlist + kConeCap;                             // sources: box row << 16 | box x
    float *s_e = reinterpret_cast<float *>(s_key + kMaxSrcF3);
    int *so = reinterpret_cast<int *>(s_e + kMaxSrcF3);        // per-plane offsets, npl + 2
    __shared__ int s_abort, s_nbin, s_l1;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = CONES ? kAllT : kFT;

    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {
        for (int s = 0; s < kR0; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        s_abort = 0;
        s_l1 = l1_lo - 1;                                      // no level-1 plane published yet
    }
    // point sources of the level-1 region (box rows 2 .. L1R + 1, all columns,
    // planes l1_lo .. l1_hi), grouped by plane: plane p's entries end up in
    // [so[p - l1_lo], so[p - l1_lo + 1])
    for (int k = tid; k < npl + 2; k += nthr) so[k] = 0;
    __syncthreads();
    const long long n_cells = (long long)f.nx * f.ny * f.nz;
    auto src_box = [&](int s, int &pl, int &key) {
        const long long c = A.src_cell[s];
        if (c < 0 || c >= n_cells) {
            if (box == 0) flag_status(A.status, kStatusBounds);
            return false;
        }
        const int cx = (int)(c % f.nx), cy = (int)((c / f.nx) % f.ny), cz = (int)(c / ((long long)f.nx * f.ny));
        const int bx = cx - ox, br = cy - oy;
        if (bx < 0 || bx >= kW || br < 2 || br >= 2 + L1R || cz < l1_lo || cz > l1_hi) return false;
        pl = cz - l1_lo;
        key = (br << 16) | bx;
        return true;
    };
    for (int s = tid; s < A.n_src; s += nthr) {
        int pl, key;
        if (src_box(s, pl, key)) atomicAdd(&so[pl + 2], 1);
    }
    __syncthreads();
    if (warp == 0) {          // inclusive scan of so[2 ..]: so[p + 1] = entries of planes < p
        int carry = 0;
        for (int base = 2; base < npl + 2; base += 32) {
            const int k = base + lane;
            int x = k < npl + 2 ? so[k] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += y;
            }
            if (k < npl + 2) so[k] = carry + x;
            carry += __shfl_sync(kFull, x, 31);
        }
    }
    __syncthreads();
    for (int s = tid; s < A.n_src; s += nthr) {
        int pl, key;
        if (src_box(s, pl, key)) {
            const int slot = atomicAdd(&so[pl + 1], 1);       // leaves so[pl + 1] = end of plane pl
            s_key[slot] = key;
            s_e[slot] = A.src_emit[s];
        }
    }

    // from here on: what earlier launches wrote (field, cone state, bins)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const unsigned plane_bytes = (unsigned)(kW * R * sizeof(float));
    auto issue = [&](int p) {
        const int s = (p - ib) % kR0;
        mbar_expect_tx(&bar[s], plane_bytes);
        tma_load_3d(P0 + s * A.p0s, &tmap, &bar[s], ox, oy, p);
    };
    if (tid == 0) {
        for (int p = ib; p < ib + kD && p <= ilast; ++p) issue(p);
        for (int p = ib + kD; p < ib + kPF && p <= ilast; ++p) tma_prefetch_3d(&tmap, ox, oy, p);
    }

    // this box's cones: the first kConeCap into shared memory, the rest keep
    // their state in global memory and their schedule word in A.sched
    if (CONES) {
        if (tid == 0) s_nbin = min(A.cnt_cur[box], A.bin_cap);
        __syncthreads();
        const int n_bin = s_nbin;
        const int *bin = A.bins_cur + (size_t)box * A.bin_cap;
        const int n = A.n;
        for (int e = tid; e < n_bin; e += nthr) {
            const int a = bin[e];
            const float pz = A.pos[2 * (size_t)n + a];
            const int w = sched_word(need_of(f, pz), 0);
            if (e < kConeCap) {
                cid[e] = a;
                cst[e] = A.pos[a];
                cst[kConeCap + e] = A.pos[(size_t)n + a];
                cst[2 * kConeCap + e] = pz;
                cst[3 * kConeCap + e] = A.dir[a];
                cst[4 * kConeCap + e] = A.dir[(size_t)n + a];
                cst[5 * kConeCap + e] = A.dir[2 * (size_t)n + a];
                csch[e] = w;
            } else {
                A.sched[a] = w;
            }
        }
    }
    __syncthreads();
    if (CONES && tid == 0) A.cnt_cur[box] = 0;       // read by every thread: free for the launch after next

    if (CONES && warp >= kFW) {
        // =================================================================== cone warps
        const int cw = warp - kFW;
        const int n_bin = s_nbin;
        const int n_sm = min(n_bin, kConeCap);
        const int n = A.n;
        int *dl = dlist + cw * (kConeCap / kCW);
        const int sy = f.nx, sz = f.nx * f.ny;
        // one sub-step on the field `F` (C^n from the input buffer for sub-step 0, C^{n+1}
        // from the scratch copy for sub-step 1, read from L2: this box's field warps stored
        // it); the footprint loads go through one base pointer at the cone's cell and
        // 32-bit offsets. Called by whole warps (the active count is a vote).
        auto step = [&](bool live, int a, int j, int prog, float *p, float *d) {
            count_active(A.counter, live);
            if (!live) return false;
            float xi[3];
            cone_noise<3>(A.c.key0, A.c.key1, (uint32_t)a, A.step0 + j, xi);
            int lo[3];
            float fr[3];
            cell_of<3>(f, p, lo, fr);
            const float *F = (j == 0 ? A.Cin : A.inter) + ((size_t)lo[2] * f.ny + lo[1]) * f.nx + lo[0];
            if (j == 1) {        // the footprint lies in the level-1 nodes this box stored and published
                const int xa = max(lo[0] - 1, 0) - ox, xb = min(lo[0] + 2, f.nx - 1) - ox;
                const int ya = max(lo[1] - 1, 0) - oy, yb = min(lo[1] + 2, f.ny - 1) - oy;
                const int za = max(lo[2] - 1, 0), zb = min(lo[2] + 2, f.nz - 1);
                if (!(xa >= 1 && xb < kW - 1 && ya >= 2 && yb < 2 + L1R && za >= l1_lo && zb <= min(prog, l1_hi)))
                    flag_status(A.status, kStatusBounds);   // never, when the schedule is right
            }
            auto ld = [&](int gi, int gj, int gk) {
                const int off = (gk - lo[2]) * sz + (gj - lo[1]) * sy + (gi - lo[0]);
                return j == 0 ? __ldg(F + off) : __ldcg(F + off);
            };
            return cone_step_rule<3>(f, A.c, ld, xi, p, d, A.src_xyz, A.n_src, A.n_stop);
        };
        auto finish = [&](int a, const float *p, const float *d, bool alive) {
            for (int k = 0; k < 3; ++k) {
                A.pos[(size_t)k * n + a] = p[k];
                A.dir[(size_t)k * n + a] = d[k];
            }
            if (!alive) {
                A.active[a] = 0;
            } else if (A.cnt_next) {
                const int bx = box_of3(A, p);
                const int slot = atomicAdd(&A.cnt_next[bx], 1);
                if (slot < A.bin_cap) A.bins_next[(size_t)bx * A.bin_cap + slot] = a;
                else flag_status(A.status, kStatusBounds);
            }
        };
        // a ready cone, with its state in registers: its next sub-step; returns the
        // cone's new schedule word (kSchedDone once both are taken or it stopped)
        auto advance = [&](bool live, int a, int wd, int prog, float *p, float *d) {
            const int j = wd >> 24;
            const bool alive = step(live, a, j, prog, p, d);
            if (!live) return kSchedDone;
            bool bad = false;
            for (int k = 0; k < 3; ++k)
                bad |= !(fabsf(p[k]) <= 3.402823466e38f) || !(fabsf(d[k]) <= 3.402823466e38f);
            if (bad) flag_status(A.status, kStatusNonFinite);
            if (alive && j == 0) return sched_word(need_of(f, p[2]), 1);
            finish(a, p, d, alive);
            return kSchedDone;
        };

        int last = -(1 << 30);
        int final_scans = 0;
        long long spins = 0;
        for (;;) {
            // the march's progress, read once per warp
            int prog = 0, ab = 0;
            if (lane == 0) {
                prog = ld_acquire(&s_l1);
                ab = *reinterpret_cast<volatile int *>(&s_abort);
            }
            prog = __shfl_sync(kFull, prog, 0);
            ab = __shfl_sync(kFull, ab, 0);
            if (ab) return;
            const bool done = prog >= l1_hi;
            if (!done && prog < last + kScanStep) {       // let the march move on
                if (++spins > kSpinLimit) {
                    if (lane == 0) flag_status(A.status, kStatusTimeout);
                    return;
                }
                __nanosleep(256);
                continue;
            }
            last = prog;
            // shared-memory cones of this warp (entries cw, cw + kCW, ...) that are ready
            int nd = 0;
            bool waiting = false;
            for (int u0 = 0; cw + kCW * u0 < n_sm; u0 += 32) {
                const int e = cw + kCW * (u0 + lane);
                const int wd = e < n_sm ? csch[e] : kSchedDone;
                const bool hit = sched_ready(wd, prog);
                waiting |= wd >= 0 && !hit;
                const unsigned m = __ballot_sync(kFull, hit);
                if (hit) dl[nd + __popc(m & ((1u << lane) - 1u))] = e;
                nd += __popc(m);
            }
            __syncwarp();
            for (int base = 0; base < nd; base += 32) {
                const bool live = base + lane < nd;
                const int e = live ? dl[base + lane] : 0;
                float p[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f};
                int a = 0, wd = 0;
                if (live) {
                    a = cid[e];
                    wd = csch[e];
                    for (int k = 0; k < 3; ++k) {
                        p[k] = cst[k * kConeCap + e];
                        d[k] = cst[(3 + k) * kConeCap + e];
                    }
                }
                const int nw = advance(live, a, wd, prog, p, d);
                if (live) {
                    csch[e] = nw;
                    waiting |= nw != kSchedDone;
                    if (nw != kSchedDone)
                        for (int k = 0; k < 3; ++k) {
                            cst[k * kConeCap + e] = p[k];
                            cst[(3 + k) * kConeCap + e] = d[k];
                        }
                }
            }
            // cones past the shared-memory slots: schedule word and state in global memory
            if (n_bin > kConeCap) {
                const int *bin = A.bins_cur + (size_t)box * A.bin_cap;
                for (int u0 = 0; kConeCap + cw + kCW * u0 < n_bin; u0 += 32) {
                    const int e = kConeCap + cw + kCW * (u0 + lane);
                    const int a = e < n_bin ? bin[e] : 0;
                    const int wd = e < n_bin ? A.sched[a] : kSchedDone;
                    const bool hit = sched_ready(wd, prog);
                    waiting |= wd >= 0 && !hit;
                    if (!__any_sync(kFull, hit)) continue;
                    float p[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f};
                    if (hit)
                        for (int k = 0; k < 3; ++k) {
                            p[k] = A.pos[(size_t)k * n + a];
                            d[k] = A.dir[(size_t)k * n + a];
                        }
                    const int nw = advance(hit, a, wd, prog, p, d);
                    if (hit) {
                        A.sched[a] = nw;
                        waiting |= nw != kSchedDone;
                        if (nw != kSchedDone)
                            for (int k = 0; k < 3; ++k) {
                                A.pos[(size_t)k * n + a] = p[k];
                                A.dir[(size_t)k * n + a] = d[k];
                            }
                    }
                }
            }
            const bool any_waiting = __any_sync(kFull, waiting);
            if (done) {
                // every footprint is published by now: a cone still waiting has just taken
                // sub-step 0 and takes sub-step 1 in the next scan, so two scans finish all
                if (!any_waiting) return;
                if (++final_scans > 2) {
                    if (lane == 0) flag_status(A.status, kStatusBounds);
                    return;
                }
            }
        }
    }

    // ======================================================================= field warps
    // a thread's level-1 groups: k = tid + m kFT -> row r1 = k / 34 (box row r1 + 2), group c = k % 34;
    // groups past the last (k >= nL1) read row 2, group 0 and store nothing
    int so0[kItems], so1[kItems], io[kItems];          // offsets: input plane, level-1 plane, grid plane
    unsigned fl[kItems];                                // flag bits, below
    constexpr unsigned kVal = 1, kIn2 = 2, kIng = 4, kWl = 8, kWr = 16, kYl = 32, kYh = 64, kE0 = 128, kE1 = 256;
    float4 a1[kItems], b3[kItems], b2[kItems];       // own nodes: input plane i - 1; level-1 planes i - 3, i - 2
#pragma unroll
    for (int m = 0; m < kItems; ++m) {
        const int k = tid + m * kFT;
        const bool v = k < nL1;
        const int r = v ? k / kW4 : 0, c = v ? k % kW4 : 0;
        const int gx = ox + 4 * c, gy = oy + r + 2;
        so0[m] = (r + 2) * kW4 + c;
        so1[m] = r * kW4 + c;
        const bool ing = v && gx >= 0 && gx < f.nx && gy >= 0 && gy < f.ny;
        io[m] = ing ? gy * f.nx + gx : 0;
        fl[m] = (v ? kVal : 0u) | ((v && r >= 2 && r < TY + 2 && c >= 1 && c <= kW4 - 2) ? kIn2 : 0u) |
                (ing ? kIng : 0u) | (gx == 0 ? kWl : 0u) | (gx + 3 == f.nx - 1 ? kWr : 0u) |
                (gy == 0 ? kYl : 0u) | (gy == f.ny - 1 ? kYh : 0u) | (c == 0 ? kE0 : 0u) |
                (c == kW4 - 1 ? kE1 : 0u);
        a1[m] = b3[m] = b2[m] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float4 *P04 = reinterpret_cast<const float4 *>(P0);
    float4 *P14 = reinterpret_cast<float4 *>(P1);
    const int p0s4 = A.p0s / 4, p1s4 = A.p1s / 4;
    const float2 alpha2 = make_float2(f.alpha, f.alpha), beta2 = make_float2(f.beta, f.beta);
    const size_t plane = (size_t)f.nx * f.ny;
    bool bad = false;

    for (int i = ib; i <= iend; ++i) {
        // the slot of plane i + kD held plane i - 3, read last in iteration i - 2 (before the
        // barrier of iteration i - 1)
        if (tid == 0) {
            if (i + kD <= ilast) issue(i + kD);
            if (i + kPF <= ilast) tma_prefetch_3d(&tmap, ox, oy, i + kPF);
        }
        const bool has_in = i <= ilast;
        bool tmo = false;
        if (has_in) {
            const int k = i - ib;
            tmo = !warp_wait_plane(&bar[k % kR0], (unsigned)((k / kR0) & 1), lane);
        }
        // ---- level 1, plane i - 1 (from input planes i - 2, i - 1, i)
        const int p1 = i - 1;
        const bool do1 = p1 >= l1_lo && p1 <= l1_hi;
        float4 nw[kItems];
        if (do1) {
            const float4 *Pn = P04 + ((i - ib) % kR0) * p0s4;
            const float4 *Pc4 = P04 + ((p1 - ib) % kR0) * p0s4;
            // input plane i - 2: its slot is reissued (plane i + 3) only after this iteration's barrier
            const float4 *Pm4 = P04 + ((p1 - 1 - ib + kR0) % kR0) * p0s4;
            const float *Pc = reinterpret_cast<const float *>(Pc4);
            float4 *Q = P14 + (p1 % kR1) * p1s4;
            const int sb = so[p1 - l1_lo], se = so[p1 - l1_lo + 1];
            const bool zlo = p1 == 0, zhi = p1 == f.nz - 1;
            float *G = CONES ? A.inter + (size_t)p1 * plane : nullptr;
            const float *Mp = MAP ? A.M + (size_t)p1 * plane : nullptr;
#pragma unroll
            for (int m = 0; m < kItems; ++m) {
                const unsigned F = fl[m];
                const float4 an = has_in ? Pn[so0[m]] : a1[m];
                const float4 c = a1[m];          // own node, input plane i - 1 (kept since the last iteration)
                float4 ym = Pc4[so0[m] - kW4];
                float4 yp = Pc4[so0[m] + kW4];
                const float4 zm = zlo ? c : Pm4[so0[m]];
                const float4 zp = zhi ? c : an;
                float xl = __shfl_up_sync(kFull, c.w, 1);
                float xr = __shfl_down_sync(kFull, c.x, 1);
                if (lane == 0 && !(F & kE0)) xl = Pc[4 * so0[m] - 1];
                if (lane == 31 && !(F & kE1)) xr = Pc[4 * so0[m] + 4];
                if (F & (kE0 | kWl)) xl = c.x;         // x wall, or outside the box (any finite value)
                if (F & (kE1 | kWr)) xr = c.w;
                if (F & kYl) ym = c;
                if (F & kYh) yp = c;
                float4 o = node_update3_x4(c, xl, xr, ym, yp, zm, zp, alpha2, beta2);
                if (MAP && (F & kIng)) {
                    const float4 mv = __ldg(reinterpret_cast<const float4 *>(Mp + io[m]));
                    o.x = fmaf(f.dt, mv.x, o.x);
                    o.y = fmaf(f.dt, mv.y, o.y);
                    o.z = fmaf(f.dt, mv.z, o.z);
                    o.w = fmaf(f.dt, mv.w, o.w);
                }
                for (int s = sb; s < se; ++s) {
                    const int key = s_key[s];
                    if ((key >> 16) * kW4 + ((key & 0xFFFF) >> 2) == so0[m]) add_comp(o, key & 3, s_e[s]);
                }
                if (F & kVal) Q[so1[m]] = o;
                // the scratch copy for the cones: every valid level-1 node inside the grid
                // (box columns 1 .. 134; the outermost node of each edge group is not valid)
                if (CONES && (F & kIng)) {
                    float *q = G + io[m];
                    if (F & kE0) {
                        q[1] = o.y;
                        q[2] = o.z;
                        q[3] = o.w;
                    } else if (F & kE1) {
                        q[0] = o.x;
                        q[1] = o.y;
                        q[2] = o.z;
                    } else {
                        *reinterpret_cast<float4 *>(q) = o;
                    }
                }
                nw[m] = o;
                a1[m] = an;                      // own input plane for the next level-1 plane
            }
        } else {
            const float4 *Pn = P04 + ((i - ib) % kR0) * p0s4;
#pragma unroll
            for (int m = 0; m < kItems; ++m) {
                a1[m] = has_in ? Pn[so0[m]] : a1[m];
                nw[m] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (CONES && do1) __threadfence_block();       // the scratch stores before the publication
        // level-1 plane i - 1 complete; a timed-out input wait aborts the whole CTA
        if (field_sync_or(tmo)) {
            if (tid == 0) {
                *reinterpret_cast<volatile int *>(&s_abort) = 1;
                flag_status(A.status, kStatusTimeout);
                for (int p = i; p <= min(i + kD, ilast); ++p) {      // let in-flight copies land (bounded)
                    const int k = p - ib;
                    mbar_wait_bounded(&bar[k % kR0], (unsigned)((k / kR0) & 1));
                }
            }
            return;
        }
        if (CONES && do1 && tid == 0) st_release(&s_l1, p1);   // cones may read level-1 planes <= p1
        // ---- level 2, plane i - 2 of the interior (from level-1 planes i - 3, i - 2, i - 1)
        const int p2 = i - 2;
        if (p2 >= zs && p2 < ze) {
            const float4 *Q4 = P14 + (p2 % kR1) * p1s4;
            const float *Qc = reinterpret_cast<const float *>(Q4);
            const int sb = so[p2 - l1_lo], se = so[p2 - l1_lo + 1];
            const bool zlo = p2 == 0, zhi = p2 == f.nz - 1;
            float *Out = A.Cout + (size_t)p2 * plane;
            const float *Mp = MAP ? A.M + (size_t)p2 * plane : nullptr;
#pragma unroll
            for (int m = 0; m < kItems; ++m) {
                const unsigned F = fl[m];
                const float4 c = b2[m];
                const bool in2 = F & kIn2;
                float4 ym = in2 ? Q4[so1[m] - kW4] : c;
                float4 yp = in2 ? Q4[so1[m] + kW4] : c;
                const float4 zm = zlo ? c : b3[m];
                const float4 zp = zhi ? c : nw[m];
                float xl = __shfl_up_sync(kFull, c.w, 1);
                float xr = __shfl_down_sync(kFull, c.x, 1);
                if (in2 && (F & kIng)) {
                    if (lane == 0) xl = Qc[4 * so1[m] - 1];
                    if (lane == 31) xr = Qc[4 * so1[m] + 4];
                    if (F & kWl) xl = c.x;
                    if (F & kWr) xr = c.w;
                    if (F & kYl) ym = c;
                    if (F & kYh) yp = c;
                    float4 o = node_update3_x4(c, xl, xr, ym, yp, zm, zp, alpha2, beta2);
                    if (MAP) {
                        const float4 mv = __ldg(reinterpret_cast<const float4 *>(Mp + io[m]));
                        o.x = fmaf(f.dt, mv.x, o.x);
                        o.y = fmaf(f.dt, mv.y, o.y);
                        o.z = fmaf(f.dt, mv.z, o.z);
                        o.w = fmaf(f.dt, mv.w, o.w);
                    }
                    for (int s = sb; s < se; ++s) {
                        const int key = s_key[s];
                        if ((key >> 16) * kW4 + ((key & 0xFFFF) >> 2) == so0[m]) add_comp(o, key & 3, s_e[s]);
                    }
                    bad |= !finite4(o);
                    *reinterpret_cast<float4 *>(Out + io[m]) = o;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < kItems; ++m) {
            b3[m] = b2[m];
            b2[m] = nw[m];
        }
    }
    if (__any_sync(kFull, bad) && lane == 0) flag_status(A.status, kStatusNonFinite);
}

// Start of a run: every active cone into its box's bin.
__global__ void bin3_kernel(F3Args A)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.n || !A.active[a]) return;
    const float p[3] = {A.pos[a], A.pos[(size_t)A.n + a], A.pos[2 * (size_t)A.n + a]};
    const int bx = box_of3(A, p);
    const int slot = atomicAdd(&A.cnt_next[bx], 1);
    if (slot < A.bin_cap) A.bins_next[(size_t)bx * A.bin_cap + slot] = a;
    else flag_status(A.status, kStatusBounds);
}

// ---------------------------------------------------------------- host side
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn_f3()
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

int plane0_stride(int TY) { return ((kW * (TY + 2 * kH) + 31) / 32) * 32; }   // 128-byte aligned slots
int plane1_stride(int TY) { return kW * (TY + 5); }

size_t smem_bytes_f3(int TY, int ZC)
{
    const int npl = ZC + 5;
    return 128 + sizeof(float) * ((size_t)kR0 * plane0_stride(TY) + (size_t)kR1 * plane1_stride(TY)) +
           (size_t)kConeCap * (6 * sizeof(float) + 3 * sizeof(int)) + (size_t)kMaxSrcF3 * 8 +
           sizeof(int) * (size_t)(npl + 2);
}

size_t smem_bytes_f3(const Fused3Geom &g) { return smem_bytes_f3(g.TY, g.ZC); }

}  // namespace

bool fused3d_geometry(const cue_params &p, Fused3Geom &g)
{
    if (p.dim != 3 || p.nx % 4 != 0 || p.nx < 4 || p.ny < 2 || p.nz < 2) return false;
    const int ntx = (p.nx + kTX - 1) / kTX;
    double best = 0.0;
    bool found = false;
    for (int TY = kMinTY; TY <= kMaxTY; ++TY) {
        const int nty = (p.ny + TY - 1) / TY;
        const long long cols = (long long)ntx * nty;
        // the last tile row and the last chunk hold at least two nodes, so a cone clamped
        // onto the far wall (cell N - 2) still lies in its box's interior rows / planes
        if (p.ny - (nty - 1) * TY < 2) continue;
        for (int c = 1; c <= p.nz; ++c) {
            const int ZC = (p.nz + c - 1) / c;
            if ((p.nz + ZC - 1) / ZC != c || p.nz - (c - 1) * ZC < 2) continue;
            const long long boxes = cols * c;
            if (boxes > (1 << 20) || smem_bytes_f3(TY, ZC) > kSmemPerCta) continue;
            const long long waves = (boxes + kSmsGB300 * kCtasPerSm - 1) / (kSmsGB300 * kCtasPerSm);
            // per box: the planes marched (chunk plus the z reach on each side) times the
            // float4 groups the two levels compute per plane
            const int planes = std::min(ZC + 6, p.nz + 2);
            const double cost = (double)waves * planes * (kW4 * (TY + 5) + (kW4 - 2) * TY);
            if (!found || cost < best * (1.0 - 1e-12)) {
                best = cost;
                found = true;
                g.TY = TY;
                g.ntx = ntx;
                g.nty = nty;
                g.nchunk = c;
                g.ZC = ZC;
                g.boxes = (int)boxes;
            }
        }
    }
    return found;
}

bool fused3d_supported(const Sim &s)
{
    if (s.fd.dim != 3 || !s.vec4 || s.n_src > kMaxSrcF3 || s.cd.steer != 0) return false;
    if (s.n_axons > 0 && !(s.cd.step_len <= s.fd.h)) return false;    // the halo covers one cell of drift
    if (!encode_fn_f3()) return false;
    Fused3Geom g;
    if (!fused3d_geometry(s.params, g)) return false;
    if (g.boxes != s.wl.n_tiles) return false;
    if (s.n_axons > 0 && s.wl.bin_cap < s.n_axons) return false;     // a bin must hold every cone of its box
    if (s.n_axons > 0 && !s.inter3()) return false;
    return true;
}

static int prepare_f3(Sim &s)
{
    if (s.geom3_ready) return CUE_OK;
    Fused3Geom g;
    if (!fused3d_geometry(s.params, g)) return CUE_ERR_ARG;
    EncodeTiledFn fn = encode_fn_f3();
    if (!fn) return CUE_ERR_CUDA;
    for (int b = 0; b < 2; ++b) {
        cuuint64_t dims[3] = {(cuuint64_t)s.fd.nx, (cuuint64_t)s.fd.ny, (cuuint64_t)s.fd.nz};
        cuuint64_t strides[2] = {(cuuint64_t)s.fd.nx * sizeof(float), (cuuint64_t)s.fd.nx * s.fd.ny * sizeof(float)};
        cuuint32_t boxd[3] = {(cuuint32_t)kW, (cuuint32_t)(g.TY + 2 * kH), 1};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = fn(reinterpret_cast<CUtensorMap *>(s.tmap3b[b]), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, s.field[b],
                        dims, strides, boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return CUE_ERR_CUDA;
    }
    const int smem = (int)smem_bytes_f3(g);
    if (cudaFuncSetAttribute(fused3d_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(fused3d_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(fused3d_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(fused3d_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess)
        return CUE_ERR_CUDA;
    // two CTAs per SM: the whole carve-out as shared memory
    if (cudaFuncSetAttribute(fused3d_kernel<false, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaFuncSetAttribute(fused3d_kernel<true, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaFuncSetAttribute(fused3d_kernel<false, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaFuncSetAttribute(fused3d_kernel<true, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return CUE_ERR_CUDA;
    s.geom3 = g;
    s.geom3_ready = true;
    return CUE_OK;
}

static F3Args make_args(Sim &s, bool cones)
{
    const Fused3Geom &g = s.geom3;
    const int r = (int)(s.bin_round & 1), rn = r ^ 1;
    F3Args A{};
    A.f = s.fd;
    A.c = s.cd;
    A.TY = g.TY;
    A.ntx = g.ntx;
    A.nty = g.nty;
    A.ZC = g.ZC;
    A.p0s = plane0_stride(g.TY);
    A.p1s = plane1_stride(g.TY);
    A.Cin = s.field[s.cur];
    A.inter = s.inter3();
    A.Cout = s.field[s.cur ^ 1];
    A.M = s.src_map;
    A.step0 = (uint32_t)s.field_step;
    A.n = s.n_axons;
    A.pos = s.pos;
    A.dir = s.dir;
    A.active = s.active;
    A.bin_cap = s.wl.bin_cap;
    A.cnt_cur = s.bin_count() + r * s.wl.n_tiles;
    A.bins_cur = s.bin_list() + (size_t)r * s.wl.n_tiles * s.wl.bin_cap;
    A.cnt_next = cones ? s.bin_count() + rn * s.wl.n_tiles : nullptr;
    A.bins_next = s.bin_list() + (size_t)rn * s.wl.n_tiles * s.wl.bin_cap;
    A.sched = reinterpret_cast<int *>(s.spill());
    A.src_cell = s.src_cell;
    A.src_emit = s.src_emit;
    A.n_src = s.n_src;
    A.src_xyz = s.src_xyz();
    A.n_stop = (s.cd.stop_r2 >= 0.0f && s.n_src > 0) ? s.n_src : 0;
    A.status = s.status();
    A.counter = s.cone_counter();
    return A;
}

// Every active cone into the current round's bins; both rounds' counts start at zero.
static cudaError_t launch_bin3(Sim &s)
{
    cudaError_t e = cudaMemsetAsync(s.bin_count(), 0, sizeof(int) * 2 * s.wl.n_tiles, s.stream);
    if (e != cudaSuccess) return e;
    F3Args A = make_args(s, true);
    // the binning kernel fills "next": point it at the current round
    const int r = (int)(s.bin_round & 1);
    A.cnt_next = s.bin_count() + r * s.wl.n_tiles;
    A.bins_next = s.bin_list() + (size_t)r * s.wl.n_tiles * s.wl.bin_cap;
    bin3_kernel<<<(s.n_axons + 255) / 256, 256, 0, s.stream>>>(A);
    s.launches++;
    return cudaGetLastError();
}

// One launch: two coupled steps (cones on) or two field steps, s.cur -> s.cur ^ 1.
static cudaError_t launch_f3(Sim &s, bool cones)
{
    const bool with_cones = cones && s.n_axons > 0;
    F3Args A = make_args(s, with_cones);
    const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(s.tmap3b[s.cur]);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)s.geom3.boxes);
    cfg.blockDim = dim3(with_cones ? kAllT : kFT);
    cfg.dynamicSmemBytes = smem_bytes_f3(s.geom3);
    cfg.stream = s.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    timing_begin(s);
    cudaError_t e;
    if (s.src_map)
        e = with_cones ? cudaLaunchKernelEx(&cfg, fused3d_kernel<true, true>, *map, A)
                       : cudaLaunchKernelEx(&cfg, fused3d_kernel<true, false>, *map, A);
    else
        e = with_cones ? cudaLaunchKernelEx(&cfg, fused3d_kernel<false, true>, *map, A)
                       : cudaLaunchKernelEx(&cfg, fused3d_kernel<false, false>, *map, A);
    timing_end(s);
    s.launches++;
    if (with_cones) s.bin_round++;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// The one-launch-per-step 3D step for the odd last step of a run.
static int single_step3(Sim &s, bool cones)
{
    float *in = s.field[s.cur], *out = s.field[s.cur ^ 1];
    bool cd = false, sd = false;
    cudaError_t e;
    if (cones) {
        if (!field3d_tma_prepare(s)) return CUE_ERR_CUDA;
        timing_begin(s);
        e = launch_field3d_tma(s, s.cur, out, &cd, &sd);
        timing_end(s);
        s.launches++;
        if (e == cudaSuccess && !cd) e = launch_cone_step(s, in, (uint32_t)s.cone_step);
        if (e == cudaSuccess && !sd) e = launch_sources(s, out);
    } else {
        e = launch_field_and_sources(s, in, out);
    }
    if (e != cudaSuccess) return CUE_ERR_CUDA;
    s.cur ^= 1;
    s.field_step++;
    if (cones) s.cone_step++;
    return CUE_OK;
}

int run_fused3d_if_supported(Sim &s, int nsteps, bool cones)
{
    if (s.fd.dim != 3) return 1;
    // only when asked for (CUE_PATH_FUSED, or a temporal depth of 2): on GB300 this path
    // measured slower than one launch per step (its march is bound by the SM's issue
    // rate and its cones by the scratch copy), so AUTO keeps the one-step kernel
    const bool asked = s.path == CUE_PATH_FUSED || (s.path == CUE_PATH_AUTO && s.temporal_depth == 2);
    if (!asked) return 1;
    if (!fused3d_supported(s)) return s.path == CUE_PATH_FUSED ? CUE_ERR_ARG : 1;
    int rc = prepare_f3(s);
    if (rc != CUE_OK) return s.path == CUE_PATH_FUSED ? rc : 1;
    const bool with_cones = cones && s.n_axons > 0;
    if (nsteps >= 2 && with_cones && launch_bin3(s) != cudaSuccess) return CUE_ERR_CUDA;
    while (nsteps >= 2) {
        if (launch_f3(s, cones) != cudaSuccess) return CUE_ERR_CUDA;
        s.cur ^= 1;
        s.field_step += 2;
        if (cones) s.cone_step += 2;
        nsteps -= 2;
    }
    if (nsteps == 1) {
        rc = single_step3(s, cones);
        if (rc != CUE_OK) return rc;
    }
    s.fused_used = true;
    return CUE_OK;
}

}  // namespace cue
