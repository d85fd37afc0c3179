// Batched evaluation: many frames of uneven size in one persistent launch,
// recorded once in a CUDA graph (tile-counter reset + persistent kernel)
// and replayed; the launch shape is chosen by timing candidates on the
// first batch of a given shape.
#include <cstring>
#include <new>
#include <cstdint>
#include "glint_kernels.cuh"

struct GlintContext {
    int device;
    uint32_t* counter;            // device: tile counter of the persistent kernel
    cudaStream_t capture;         // internal stream used for capture and tuning
    // tuning
    bool tuned;
    uint64_t signature;
    GlintLaunch launch;
    // graph
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaGraphNode_t kernel_node;
    int graph_variant;            // kernel variant the graph holds (kernel_variant)
    // host copies of the kernel arguments referenced by node updates
    glint::KParams P;
    glint::BatchDesc B;
};

namespace glint {
namespace {

const GlintLaunch kCandidates[] = {{512, 0}, {256, 0}, {1024, 0}, {256, 4}, {256, 8}, {512, 2}, {1024, 1}};

uint64_t batch_signature(const GlintFrame* frames, int n) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
    mix((uint64_t)n);
    for (int f = 0; f < n; ++f) {
        mix((uint64_t)frames[f].width);
        mix((uint64_t)frames[f].height);
        mix((uint64_t)frames[f].n_lights);
        mix(frames[f].mat_px ? 1u : 0u);
    }
    return h;
}

// Fill B (frames, tile offsets) for tiles of `threads` pixels.
void fill_batch(GlintContext* c, const GlintFrame* frames, int n, float* const* outs, int threads) {
    BatchDesc& B = c->B;
    B.n = n;
    B.persistent = c->launch.ctas_per_sm > 0;
    B.counter = c->counter;
    int t = 0;
    for (int f = 0; f < n; ++f) {
        B.frames[f] = make_frame_desc(&frames[f], outs[f]);
        B.tile_base[f] = t;
        t += frame_tiles(B.frames[f], threads);
    }
    B.tile_base[n] = t;
}

FwdLaunch batch_launch(const BatchDesc& B, GlintLaunch L) {
    const int sms = num_sms() > 0 ? num_sms() : 1;
    const int tiles = B.tile_base[B.n];
    if (L.ctas_per_sm == 0) return FwdLaunch{L.threads_per_cta, tiles};
    const int cap = sms * L.ctas_per_sm;
    return FwdLaunch{L.threads_per_cta, tiles < cap ? tiles : cap};
}

cudaError_t enqueue(GlintContext* c, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(c->counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    return launch_batch(c->P, c->B, s, batch_launch(c->B, c->launch));
}

// Time each candidate shape on the internal stream (blocking).
cudaError_t autotune(GlintContext* c, const GlintFrame* frames, int n, float* const* outs) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
    float best = 1e30f;
    GlintLaunch best_l = kCandidates[0];
    for (const GlintLaunch& L : kCandidates) {
        c->launch = L;
        fill_batch(c, frames, n, outs, L.threads_per_cta);
        if ((e = enqueue(c, c->capture)) != cudaSuccess) break;          // warm-up
        if ((e = cudaEventRecord(e0, c->capture)) != cudaSuccess) break;
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = enqueue(c, c->capture);
        if (e != cudaSuccess) break;
        if ((e = cudaEventRecord(e1, c->capture)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_l = L; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    c->launch = best_l;
    return cudaSuccess;
}

cudaError_t capture_graph(GlintContext* c) {
    if (c->exec) { cudaGraphExecDestroy(c->exec); c->exec = nullptr; }
    if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
    cudaError_t e = cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t ee = enqueue(c, c->capture);
    e = cudaStreamEndCapture(c->capture, &c->graph);
    if (ee != cudaSuccess) return ee;
    if (e != cudaSuccess) return e;
    if ((e = cudaGraphInstantiate(&c->exec, c->graph, 0)) != cudaSuccess) return e;
    c->graph_variant = kernel_variant(c->P);
    size_t nn = 0;
    if ((e = cudaGraphGetNodes(c->graph, nullptr, &nn)) != cudaSuccess) return e;
    cudaGraphNode_t nodes[8];
    if (nn > 8) return cudaErrorUnknown;
    if ((e = cudaGraphGetNodes(c->graph, nodes, &nn)) != cudaSuccess) return e;
    c->kernel_node = nullptr;
    for (size_t k = 0; k < nn; ++k) {
        cudaGraphNodeType t;
        cudaGraphNodeGetType(nodes[k], &t);
        if (t == cudaGraphNodeTypeKernel) c->kernel_node = nodes[k];
    }
    return c->kernel_node ? cudaSuccess : cudaErrorUnknown;
}

// Point the instantiated graph's kernel node at the current arguments.
cudaError_t update_graph(GlintContext* c) {
    const FwdLaunch cfg = batch_launch(c->B, c->launch);
    void* args[2] = {&c->P, &c->B};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(batch_kernel_fn(kernel_variant(c->P)));
    kp.gridDim = dim3(cfg.blocks);
    kp.blockDim = dim3(cfg.threads);
    kp.sharedMemBytes = (unsigned)fwd_smem_bytes(cfg.threads);
    kp.kernelParams = args;
    return cudaGraphExecKernelNodeSetParams(c->exec, c->kernel_node, &kp);
}

}  // namespace
}  // namespace glint

using namespace glint;

extern "C" {

int glint_ctx_create(GlintContext** out) {
    if (!out) return GLINT_ERR_ARG;
    *out = nullptr;
    GlintContext* c = new (std::nothrow) GlintContext;
    if (!c) return GLINT_ERR_CUDA;
    std::memset(static_cast<void*>(c), 0, sizeof(GlintContext));
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&c->counter), sizeof(uint32_t)) != cudaSuccess) {
        delete c;
        return GLINT_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(c->counter);
        delete c;
        return GLINT_ERR_CUDA;
    }
    *out = c;
    return GLINT_OK;
}

void glint_ctx_destroy(GlintContext* c) {
    if (!c) return;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->capture) cudaStreamDestroy(c->capture);
    if (c->counter) cudaFree(c->counter);
    delete c;
}

int glint_ctx_get_launch(const GlintContext* c, GlintLaunch* out) {
    if (!c || !out) return GLINT_ERR_ARG;
    if (!c->tuned) return GLINT_ERR_ARG;
    *out = c->launch;
    return GLINT_OK;
}

int glint_ctx_set_launch(GlintContext* c, const GlintLaunch* in) {
    if (!c || !in) return GLINT_ERR_ARG;
    const int t = in->threads_per_cta;
    if ((t != 128 && t != 256 && t != 512 && t != 1024) || in->ctas_per_sm < 0 || in->ctas_per_sm > 16)
        return GLINT_ERR_ARG;
    c->launch = *in;
    c->tuned = true;
    c->signature = 0;          // applies to whatever batch comes next
    return GLINT_OK;
}

int glint_eval_batch(GlintContext* c, const GlintFrame* frames, int32_t n_frames, const GlintMaterial* material,
                     const GlintLight* lights, float* const* outs, void* stream) {
    if (!c || !frames || !outs || n_frames <= 0 || n_frames > kMaxBatch) return GLINT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device) return GLINT_ERR_ARG;
    int nl_max = 0;
    long long tiles_min = 0;
    for (int f = 0; f < n_frames; ++f) {
        int rc = check_frame_shape(&frames[f], lights);
        if (rc) return rc;
        nl_max = frames[f].n_lights > nl_max ? frames[f].n_lights : nl_max;
        tiles_min += ((long long)frames[f].width * frames[f].height + 1023) / 1024;
    }
    if (tiles_min * 16 > 0x7fffffffLL) return GLINT_ERR_ARG;     // 128-pixel tiles, with 2-D padding
    int rc = make_material_params(material, lights, nl_max, &c->P);
    if (rc) return rc;
    for (int f = 0; f < n_frames; ++f) {
        if ((rc = check_frame_device(&frames[f], lights))) return rc;
        if ((rc = check_device_ptr(outs[f], 4))) return rc;
    }
    const uint64_t sig = batch_signature(frames, n_frames);
    if (!c->tuned || (c->signature != 0 && c->signature != sig)) {
        // the tuning launches run on the internal stream: order them after
        // the work already queued on the caller's stream (the inputs)
        cudaEvent_t ready;
        if ((rc = cuda_rc(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming)))) return rc;
        cudaError_t e = cudaEventRecord(ready, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->capture, ready, 0);
        cudaEventDestroy(ready);
        if ((rc = cuda_rc(e))) return rc;
        if ((rc = cuda_rc(autotune(c, frames, n_frames, outs)))) return rc;
        c->tuned = true;
        c->signature = sig;
    } else if (c->signature == 0) {
        c->signature = sig;
    }
    fill_batch(c, frames, n_frames, outs, c->launch.threads_per_cta);
    if (!c->exec || c->graph_variant != kernel_variant(c->P)) {      // a new kernel: record again
        if ((rc = cuda_rc(capture_graph(c)))) return rc;
    }
    if ((rc = cuda_rc(update_graph(c)))) return rc;
    return cuda_rc(cudaGraphLaunch(c->exec, (cudaStream_t)stream));
}

}  // extern "C"
