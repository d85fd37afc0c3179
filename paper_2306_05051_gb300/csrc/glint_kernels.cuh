// Host-side declarations shared by the library's translation units (not part
// of the public interface).
#pragma once
#include <cuda_runtime.h>
#include "glint_pixel.cuh"
#include "../../include/glint.h"

namespace glint {

// Launch configuration of the forward kernels.
struct FwdLaunch {
    int threads;
    int blocks;
};

constexpr int kMaxBatch = 128;

// Frames of one persistent batched launch (passed by value as a kernel
// parameter, so a graph node can be re-pointed without re-capture).
// Tiles of a frame for CTAs of `threads` threads: chooses F.tile_w (row tiles
// or 2-D blocks) and returns the number of tiles.
int frame_tiles(FrameDesc& F, int threads);

struct BatchDesc {
    int32_t n;
    int32_t persistent;                 // 1: CTAs take tiles from the counter; 0: CTA b shades tile b
    uint32_t* counter;                  // tile counter, zero at launch
    int32_t tile_base[kMaxBatch + 1];   // first tile of each frame; tile_base[n] = total
    FrameDesc frames[kMaxBatch];
};

// Material, lights (n of them) and tables into KParams (host only).
int make_material_params(const GlintMaterial* mat, const GlintLight* lights, int n_lights, KParams* P);
// Shape checks of a frame (host only).
int check_frame_shape(const GlintFrame* f, const GlintLight* lights);
FrameDesc make_frame_desc(const GlintFrame* f, float* out);
// Validate a frame's device pointers (null, alignment, device accessibility).
int check_frame_device(const GlintFrame* frame, const GlintLight* lights);
int check_device_ptr(const void* p, size_t align);
int num_sms();
int cuda_rc(cudaError_t e);

cudaError_t launch_fwd(const KParams& P, const FrameDesc& F, cudaStream_t s, FwdLaunch cfg);
cudaError_t launch_batch(const KParams& P, const BatchDesc& B, cudaStream_t s, FwdLaunch cfg);
// Image-kernel variants: anisotropic (ring) grids, isotropic-grid mode
// (n_rings = 0), classical sampler (sampler = 1), random-number table
// (rng_table = 1), the last three being ablations of the paper's method.
enum KernelVariant { kRing = 0, kIsoGrid = 1, kClassicalSampler = 2, kRngTable = 3, kNumVariants = 4 };
int kernel_variant(const KParams& P);
// Fill the random-number table of the current device on first use (rng_table = 1).
cudaError_t ensure_rng_table(cudaStream_t s);
const void* batch_kernel_fn(int variant);   // the batch kernel of a variant
size_t fwd_smem_bytes(int threads);
FwdLaunch default_fwd_launch(int npx);
FwdLaunch make_fwd_launch(int npx, int threads, int ctas_per_sm);
cudaError_t launch_trace(const KParams& P, const FrameDesc& F, const int32_t* px, int32_t n_px,
                         GlintTracePix* pix, GlintTraceRec* recs, int32_t cap, cudaStream_t s);

}  // namespace glint
