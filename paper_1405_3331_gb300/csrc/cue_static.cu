// cue_static.cu -- a coupled run for callers that cannot allocate device
// memory (for example code running inside another framework's allocator, or
// a host that forbids cudaMalloc after start-up).  Instead of a caller-sized
// workspace it uses one file-scope device array of fixed size as scratch.
//
// The array lives in the module image: every GPU that loads libcue.so holds
// kStaticScratchBytes for it until the process exits.  All calls on a device
// share it and it keeps the last call's contents; cue_init clears the parts
// that must start at zero (status word, cone counter, tile counts).  Calls
// whose GPU work overlaps (two streams, or two host threads) race on it.
// The status word sits at the start of the array (the workspace layout puts
// it at offset 0); cue_static_status reads and clears it.
#include "cue_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = 4u << 20;   // 4 MiB

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch in the current context.  Host code may
// not use the symbol itself: on the host it names a stand-in object, not
// device memory.  The address is looked up on every call (the lookup
// allocates nothing), so a reset device or another current context never
// sees an address resolved elsewhere.  The first lookup on a device loads the
// module there, which is why the first call must come before any stream
// capture.
int scratch_for_current_device(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return CUE_ERR_CUDA;
    *out = p;
    return CUE_OK;
}

}  // namespace

extern "C" {

size_t cue_static_scratch_bytes(void) { return kStaticScratchBytes; }

int sim_run_static(const cue_params *params, const cone_params *cone, float *d_field_a, float *d_field_b,
                   const int32_t *d_src_cell, const float *d_src_emit, int32_t n_src, const float *d_src_map,
                   float *d_pos, float *d_dir, uint8_t *d_active, int32_t n_axons, int64_t step0, int32_t nsteps,
                   void *stream, int32_t *cur_buffer_out)
{
    if (!cur_buffer_out || nsteps < 0 || step0 < 0 || step0 + nsteps > 0xFFFFFFFFLL) return CUE_ERR_ARG;
    const size_t need = cue_workspace_bytes(params, n_src, n_axons);
    if (need == 0) return CUE_ERR_ARG;
    if (need > kStaticScratchBytes) return CUE_ERR_SCRATCH;
    void *ws = nullptr;
    int rc = scratch_for_current_device(&ws);
    if (rc != CUE_OK) return rc;
    cue_sim *h = nullptr;
    rc = cue_init(&h, params, cone, d_field_a, d_field_b, d_src_cell, d_src_emit, n_src, d_src_map, d_pos, d_dir,
                  d_active, n_axons, ws, kStaticScratchBytes, stream);
    if (rc != CUE_OK) return rc;
    cue::sim_no_host_alloc(h);          // no pinned readback word: this entry point allocates nothing
    rc = cue_set_state(h, step0, step0, 0);
    if (rc == CUE_OK) rc = sim_run(h, nsteps);
    int64_t fs = 0, cs = 0;
    int32_t cur = 0;
    if (rc == CUE_OK) rc = cue_get_state(h, &fs, &cs, &cur);
    cue_destroy(h);
    if (rc == CUE_OK) *cur_buffer_out = cur;
    return rc;
}

int cue_static_status(void *stream)
{
    void *ws = nullptr;
    int rc = scratch_for_current_device(&ws);
    if (rc != CUE_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, ws, sizeof(word), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && word) {
        e = cudaMemsetAsync(ws, 0, sizeof(word), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return CUE_ERR_CUDA;
    if (word & cue::kStatusNonFinite) return CUE_ERR_NONFINITE;
    if (word & cue::kStatusTimeout) return CUE_ERR_TIMEOUT;
    if (word & cue::kStatusBounds) return CUE_ERR_BOUNDS;
    return CUE_OK;
}

}  // extern "C"
