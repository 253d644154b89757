// k_cone.cu -- one growth-cone step for every active cone (rows a3-a6) on
// the field of the current step, one thread per cone.  The field is read
// through the read-only path; source node coordinates for the stop test are
// staged in shared memory per block.
//
// Steering (Sec. 3.5, "Growth cone steering mechanisms", Eq. 6-7): vector
// addition of the previous direction, the normalised sensed cue gradient and
// Philox/Box-Muller noise (Sec. 5.1, Sec. 3.2); advance by a fixed length;
// stop outside the domain (Sec. 3.4) or near a source (Sec. 3.3).
#include "cue_internal.h"

namespace cue {
namespace {

constexpr int kMaxSmemSources = 2048;   // at most [3][2048] floats = 24 KiB of dynamic shared memory

// State is read from (pin, din) and written to (pout, dout); the coupled run
// passes the same arrays for both, the adjoint's recompute passes the next
// stored step.
template <int DIM>
__global__ void __launch_bounds__(128) cone_plain(FieldDesc f, ConeDesc c, const float *__restrict__ C,
                                                  uint32_t step, int n, const float *pin, const float *din,
                                                  float *pout, float *dout, uint8_t *__restrict__ active,
                                                  const float *__restrict__ src_xyz, int n_src,
                                                  unsigned *status, unsigned long long *counter)
{
    extern __shared__ float s_src[];         // [DIM][n_src] when the stop test is on and fits
    const bool use_stop = c.stop_r2 >= 0.0f && n_src > 0;
    const bool in_smem = n_src <= kMaxSmemSources;
    if (use_stop && in_smem) {
        for (int i = threadIdx.x; i < DIM * n_src; i += blockDim.x) s_src[i] = src_xyz[i];
        __syncthreads();
    }
    // the state loads go out together and the noise is drawn while they are in flight
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const bool inr = a < n;
    const uint8_t act = inr ? active[a] : 0;
    float p[DIM], d[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        p[i] = inr ? pin[(size_t)i * n + a] : 0.0f;
        d[i] = inr ? din[(size_t)i * n + a] : 0.0f;
    }
    float xi[DIM];
    cone_noise<DIM>(c.key0, c.key1, (uint32_t)a, step, xi);
    const bool live = inr && act;
    count_active(counter, live);
    if (!live) return;
    const size_t sy = f.nx, sz = (size_t)f.nx * f.ny;
    auto ld = [&](int i, int j, int k) { return __ldg(C + (size_t)i + sy * j + sz * k); };
    const float *src = in_smem ? s_src : src_xyz;
    const int stride = n_src;
    bool alive = cone_step_rule<DIM>(f, c, ld, xi, p, d, src, stride, use_stop ? n_src : 0);
    bool bad = false;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        pout[(size_t)i * n + a] = p[i];
        dout[(size_t)i * n + a] = d[i];
        bad |= !(fabsf(p[i]) <= 3.402823466e38f) || !(fabsf(d[i]) <= 3.402823466e38f);
    }
    if (!alive) active[a] = 0;
    if (bad) flag_status(status, kStatusNonFinite);
}

}  // namespace

cudaError_t launch_cone_step_io(Sim &s, const float *C, uint32_t step, const float *pin, const float *din,
                                float *pout, float *dout)
{
    if (s.n_axons == 0) return cudaSuccess;
    // One cone per thread; small blocks spread a few thousand cones over many SMs
    // (each cone is a short chain of dependent loads, so the more SMs the better).
    const int threads = s.n_axons >= 65536 ? 128 : 64;
    const int blocks = (s.n_axons + threads - 1) / threads;
    const bool stage = s.cd.stop_r2 >= 0.0f && s.n_src > 0 && s.n_src <= kMaxSmemSources;
    const size_t smem = stage ? sizeof(float) * s.fd.dim * s.n_src : 0;
    if (s.fd.dim == 2)
        cone_plain<2><<<blocks, threads, smem, s.stream>>>(s.fd, s.cd, C, step, s.n_axons, pin, din, pout, dout, s.active,
                                                    s.src_xyz(), s.n_src, s.status(), s.cone_counter());
    else
        cone_plain<3><<<blocks, threads, smem, s.stream>>>(s.fd, s.cd, C, step, s.n_axons, pin, din, pout, dout, s.active,
                                                    s.src_xyz(), s.n_src, s.status(), s.cone_counter());
    s.launches++;
    return cudaGetLastError();
}

cudaError_t launch_cone_step(Sim &s, const float *C, uint32_t step)
{
    return launch_cone_step_io(s, C, step, s.pos, s.dir, s.pos, s.dir);
}

}  // namespace cue
