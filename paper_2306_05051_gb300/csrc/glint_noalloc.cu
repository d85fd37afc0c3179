// Batched evaluation that allocates nothing.
//
// glint_eval_batch keeps its tile counter in device memory that
// glint_ctx_create obtains with cudaMalloc.  Some callers cannot allocate:
// for example a renderer that hands this library a fixed memory budget at
// start-up, code running where an allocation would synchronise the device in
// the middle of a frame, or a plug-in whose host application owns every
// allocation.  glint_eval_batch_noalloc serves them: the persistent batch
// kernel is unchanged, and its scratch - one tile counter per chunk of up to
// 128 frames - lives in the file-scope array below, which every GPU that
// loads the library holds from module load until the process exits.
#include <mutex>
#include "glint_kernels.cuh"

namespace glint {
namespace {

// 64 counters of 4 bytes (256 bytes): at most 64 chunks of kMaxBatch frames.
constexpr int kNoallocCounters = 64;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoallocCounters];

// Launch shape of the no-allocation path (no timing, no context).
constexpr GlintLaunch kNoallocLaunch = {256, 4};

std::mutex g_scratch_mutex;
uint32_t* g_scratch_addr[64];     // device address of the array, per device

// The array's name is only a host-side stand-in; the device address is looked
// up once per device, with that device current.
int scratch_of_current_device(uint32_t** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GLINT_ERR_CUDA;
    if (dev < 0 || dev >= 64) return GLINT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_rc(e);
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_addr[dev];
    return GLINT_OK;
}

}  // namespace
}  // namespace glint

using namespace glint;

extern "C" int glint_eval_batch_noalloc(const GlintFrame* frames, int32_t n_frames, const GlintMaterial* material,
                                        const GlintLight* lights, float* const* outs, void* stream) {
    if (!frames || !outs || n_frames <= 0) return GLINT_ERR_ARG;
    const int chunks = (n_frames + kMaxBatch - 1) / kMaxBatch;
    if (chunks > kNoallocCounters) return GLINT_ERR_WORKSPACE;
    int nl_max = 0;
    for (int f = 0; f < n_frames; ++f) {
        const int rc = check_frame_shape(&frames[f], lights);
        if (rc) return rc;
        nl_max = frames[f].n_lights > nl_max ? frames[f].n_lights : nl_max;
    }
    KParams P;
    int rc = make_material_params(material, lights, nl_max, &P);
    if (rc) return rc;
    for (int f = 0; f < n_frames; ++f) {
        if ((rc = check_frame_device(&frames[f], lights))) return rc;
        if ((rc = check_device_ptr(outs[f], 4))) return rc;
    }
    uint32_t* scratch = nullptr;
    if ((rc = scratch_of_current_device(&scratch))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the counters keep the previous call's values: clear them first
    if ((rc = cuda_rc(cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * chunks, s)))) return rc;
    const int sms = num_sms() > 0 ? num_sms() : 1;
    BatchDesc B;
    for (int c = 0; c < chunks; ++c) {
        const int f0 = c * kMaxBatch;
        const int n = n_frames - f0 < kMaxBatch ? n_frames - f0 : kMaxBatch;
        B.n = n;
        B.persistent = 1;
        B.counter = scratch + c;
        long long t = 0;
        for (int k = 0; k < n; ++k) {
            B.frames[k] = make_frame_desc(&frames[f0 + k], outs[f0 + k]);
            B.tile_base[k] = (int)t;
            t += frame_tiles(B.frames[k], kNoallocLaunch.threads_per_cta);
            if (t > 0x7fffffffLL) return GLINT_ERR_ARG;
        }
        B.tile_base[n] = (int)t;
        const int cap = sms * kNoallocLaunch.ctas_per_sm;
        const FwdLaunch cfg{kNoallocLaunch.threads_per_cta, t < cap ? (int)t : cap};
        if ((rc = cuda_rc(launch_batch(P, B, s, cfg)))) return rc;
    }
    return GLINT_OK;
}
