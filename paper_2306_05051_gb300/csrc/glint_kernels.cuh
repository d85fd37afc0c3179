// Host-side declarations shared by the library's translation units (not part
// of the public interface).
#pragma once
#include <cuda_runtime.h>
#include "glint_pixel.cuh"
#include "../../include/glint.h"

namespace glint {

// Launch configuration of the plain forward kernel.
struct FwdLaunch {
    int threads;
    int blocks;
};

// Fill every derived field of KParams from the public structs (no device work).
int make_params(const GlintFrame* frame, const GlintMaterial* mat, const GlintLight* lights, float* out,
                KParams* P);
// Validate a frame's device pointers (null, alignment, device accessibility).
int check_frame_device(const GlintFrame* frame, const GlintLight* lights);
int num_sms();

cudaError_t launch_fwd(const KParams& P, cudaStream_t s, FwdLaunch cfg);
size_t fwd_smem_bytes(int threads);
FwdLaunch default_fwd_launch(int npx);
FwdLaunch make_fwd_launch(int npx, int threads, int ctas_per_sm);
cudaError_t launch_trace(const KParams& P, const int32_t* px, int32_t n_px, GlintTracePix* pix,
                         GlintTraceRec* recs, int32_t cap, cudaStream_t s);
size_t tables_bytes(int M);

}  // namespace glint
