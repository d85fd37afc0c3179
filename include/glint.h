/*
 * glint.h - C ABI of the GB300 (sm_103a) glint BRDF library.
 *
 * The library evaluates, per pixel of a G-buffer, the glint BRDF of
 * Deliot & Belcour, "Real-Time Rendering of Glinty Appearances using
 * Distributed Binomial Laws on Anisotropic Grids" (HPG 2023):
 *   Sec. 3, Eq. 1-4  microfacet shading with the NDF replaced by a counting
 *                    process D_P = D(n)/R * b(N(P), p) / N(P), p = R D(h)/D(n);
 *   Sec. 4.2, Eq. 10 distributed binomial blending across two LODs;
 *   Sec. 5           anisotropic virtual grids (scale, ratio, orientation);
 *   Sec. 6.1-6.2     tetrahedral blending and simplex surface grids
 *                    (48 binomial evaluations per pixel and light);
 *   Sec. 6.3         gated Gaussian approximation of the binomial law.
 *
 * Conventions (all entry points):
 *   - Pointers marked "device" are CUDA device pointers owned by the caller;
 *     the library never frees them.  "host" pointers are read during the
 *     call only, unless stated otherwise.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream).  Output buffers are valid
 *     once the stream has reached the end of the enqueued work.
 *   - Return value: GLINT_OK (0) or a negative GLINT_ERR_* code; no
 *     exception crosses the interface.  Arguments are validated on the host
 *     before anything is enqueued; on error nothing is enqueued.
 *   - Pixels are row-major, x fastest.  Background pixels (normal = 0) and
 *     invalid pixels produce 0.
 */
#ifndef GLINT_H
#define GLINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GLINT_OK                   0
#define GLINT_ERR_ARG             -1  /* null pointer, bad size or parameter */
#define GLINT_ERR_ALIGN           -2  /* device pointer not 16-byte aligned */
#define GLINT_ERR_NOT_DEVICE_PTR  -3  /* pointer is not device-accessible memory */
#define GLINT_ERR_CUDA            -4  /* a CUDA runtime call failed */
#define GLINT_ERR_UNSUPPORTED     -5  /* no sm_103a device, or parameter outside supported range */
#define GLINT_ERR_WORKSPACE       -6  /* workspace or staging buffer too small */

#define GLINT_MAX_LIGHTS   8
#define GLINT_MAX_SUB      64
#define GLINT_MAX_RINGS    6
#define GLINT_MAX_LODS     16

/* Material (Sec. 3 and Sec. 5-6 parameters).
 *   ndf         0 Beckmann, 1 GGX (Sec. 7: any NDF converges).
 *   alpha_x/y   NDF roughness along tangent / bitangent (ignored when a
 *               per-pixel material plane is given).
 *   ln_density  natural log of the flake density, flakes per unit uv^2
 *               (ignored with a per-pixel plane).  Level 0 holds one flake
 *               per texel (Sec. 4.1, stratified distribution).
 *   R           Eq. 4 ratio, 0 < R <= 1 (Sec. 7 uses 0.034).
 *   F0          Schlick reflectance at normal incidence.
 *   gamma       angular texel size in projected half-vector units, >= 1e-3
 *               (Sec. 5.2, "subdivide it to account for the glints'
 *               micro-roughness").
 *   n_lods      L, 2..16 levels of detail; level l holds f^l flakes per texel.
 *   n_rings     M, 0..6 anisotropy rings; ring m has ratio 2^m and 2^(m+1)
 *               orientations (Fig. 5).  M = 0: isotropic grids only, the
 *               Sec. 4 method with the anisotropy filtered by hand - the
 *               footprint is cut along its major axis into ceil(r) pieces,
 *               each evaluated at its two LODs (24 evaluations per piece and
 *               light instead of 48).
 *   lod_factor  f, area ratio between consecutive LODs: 2 or 4 (Eq. 13 writes
 *               powers of two; Sec. 1 says consecutive LODs quadruple).
 *   max_sub     K_max, 1..64: most sub-footprints one pixel is cut into when
 *               its ratio exceeds 2^M or its area exceeds the top level.
 *   seed        32-bit seed of the per-texel hash.
 *   lod_blend   0: distributed binomial (Sec. 4.2, the paper's method): each
 *               grid vertex counts w_i N_i trials.  1: linear mix of LOD
 *               outputs (Sec. 3, "Temporal Coherence", the scheme Sec. 4.2
 *               replaces): each grid vertex counts over its whole cell and
 *               its count is weighted by w_i (same mean, smaller variance).
 *   sampler     0: gated Gaussian approximation (Sec. 6.3, the paper's).
 *               1: classical approximation (Sec. 6.3, the one it replaces):
 *               a floored Gaussian of mean N p and variance N p (1 - p)
 *               sampled at the first hash word where N p > 5 or N > 16, else
 *               an explicit sum of ceil(N) Bernoulli trials (the last one of
 *               weight N - floor N) whose uniforms are fmix32(h1 + k
 *               0x9E3779B9), k = 1..ceil N, of the second word h1.
 *   rng_table   0: the two uniforms of an evaluation come from mixing its
 *               spatial and angular hash words (fmix32).  1: they are fetched
 *               from a precomputed table of 2^16 word pairs (Sec. 6.3, last
 *               paragraph: a small texture of random numbers), entry
 *               (s + a) >> 16 of the spatial and angular words; requires
 *               n_rings > 0 and sampler = 0 (else GLINT_ERR_UNSUPPORTED).  The
 *               table lives in static device memory of the library, filled
 *               by the first call that uses it on a device (one kernel and a
 *               wait for it on the call's stream): make that first call
 *               before any stream capture.
 *               lod_blend = 1, sampler = 1 and rng_table = 1 are ablations:
 *               glint_eval, glint_eval_batch and glint_eval_trace accept
 *               them; glint_backward and glint_fit_l2 return
 *               GLINT_ERR_UNSUPPORTED. */
typedef struct GlintMaterial {
    int32_t  ndf;
    float    alpha_x, alpha_y;
    float    ln_density;
    float    R;
    float    F0;
    float    gamma;
    int32_t  n_lods;
    int32_t  n_rings;
    int32_t  lod_factor;
    int32_t  max_sub;
    uint32_t seed;
    int32_t  lod_blend;
    int32_t  sampler;
    int32_t  rng_table;
} GlintMaterial;

/* Punctual light (Sec. 8: point lights only; cost linear in lights).
 *   kind 0: point light; direction (towards the light) and irradiance-scaled
 *           intensity E are read per pixel from the frame's light plane.
 *   kind 1: directional light; dir (towards the light, any length > 0) and
 *           intensity apply to every pixel. */
typedef struct GlintLight {
    int32_t kind;
    float   dir[3];
    float   intensity;
} GlintLight;

/* One frame of G-buffer, all planes device pointers, 16-byte aligned.
 *   gbuf      [height][width][16] float: u, v, du/dx, dv/dx, du/dy, dv/dy,
 *             n.xyz, t.xyz, towards-viewer.xyz, 0.  n = 0 marks background.
 *   light_px  [n_lights][height][width][4] float: per-pixel (direction to the
 *             light xyz, E) for lights of kind 0; may be NULL when every light
 *             is directional.
 *   mat_px    [height][width][2] float: per-pixel (alpha, flakes per uv^2),
 *             isotropic alpha; NULL to use the scalar material. */
typedef struct GlintFrame {
    const float* gbuf;
    const float* light_px;
    const float* mat_px;
    int32_t width, height;
    int32_t n_lights;
} GlintFrame;

/* Human-readable text of an error code (static string). */
const char* glint_error_string(int code);

/* Library version, major * 10000 + minor * 100 + patch. */
int glint_version(void);

/* Plain forward evaluation of one frame (Sec. 3-6, whole hot path):
 * out[y][x] = sum over lights of F G D_P E / (4 <n.w_v>).
 *   out: device, [height][width] float, written completely.
 * Errors: GLINT_ERR_ARG (null, sizes <= 0, width*height > 2^31-1,
 * n_lights out of [0, 8], light_px NULL with a kind-0 light, material out of
 * range), GLINT_ERR_ALIGN, GLINT_ERR_NOT_DEVICE_PTR, GLINT_ERR_CUDA. */
int glint_eval(const GlintFrame* frame, const GlintMaterial* material,
               const GlintLight* lights, float* out, void* stream);

/* Launch shape of the forward kernel: threads per CTA (128, 256, 512 or
 * 1024; one warp shades 32 pixels, a CTA a tile of that many consecutive
 * pixels) and CTAs per SM.  ctas_per_sm = 0 (glint_eval's default, with 512
 * threads): one CTA per tile, the hardware scheduler balances tiles of
 * uneven cost over the SMs.  ctas_per_sm = 1..16: a persistent grid of
 * min(tiles, SMs x ctas_per_sm) CTAs loops over the tiles (the batched
 * path's CTAs then take tiles from the context's counter). */
typedef struct GlintLaunch {
    int32_t threads_per_cta;
    int32_t ctas_per_sm;
} GlintLaunch;

/* glint_eval with an explicit launch shape (used by the autotuner).  Same
 * result bits as glint_eval for every shape. */
int glint_eval_launch(const GlintFrame* frame, const GlintMaterial* material,
                      const GlintLight* lights, float* out, const GlintLaunch* launch, void* stream);

/* The same evaluation with host buffers: copies every plane of `frame`
 * (host pointers, ideally pinned) into `staging` (device, caller-owned, at
 * least glint_eval_host_staging_size() bytes), evaluates, and copies the
 * image back to `out` (host).  The frame is processed in bands of about 0.5 M
 * pixels of whole rows (at most 64 bands) so that copies in, kernels and
 * copies out of different bands overlap: the copies run on two internal
 * streams of the library (one pair per device, created on first use) that
 * fork from and join back into `stream` through events.  Work enqueued on
 * `stream` after the call sees the finished image; the caller synchronises
 * `stream` before reading `out`.  Same image bits as glint_eval. */
size_t glint_eval_host_staging_size(int32_t width, int32_t height, int32_t n_lights,
                                    int32_t has_light_plane, int32_t has_material_plane);
int glint_eval_host(const GlintFrame* host_frame, const GlintMaterial* material,
                    const GlintLight* lights, float* out_host,
                    void* staging, size_t staging_bytes, void* stream);

/* Batched evaluation: many frames (each with its own planes, size and
 * n_lights; one material and one light array for all) shaded by ONE
 * launch over the concatenated tiles of all frames - persistent CTAs taking
 * 1-tile work items from a counter, or one CTA per tile, whichever the tuner
 * finds faster - so frames of uneven size and cost balance across the GPU.
 * The launch is recorded in a CUDA graph (counter reset + kernel) owned by
 * the context and replayed on later calls; a new set of frame pointers only
 * updates the graph's kernel node (a switch between n_rings = 0 and > 0
 * records it again).  Results are bit-identical to glint_eval per frame.
 *
 * Context: created on the current device; owns a 4-byte device counter, an
 * internal stream and the graph.  Not thread-safe; batches of one context
 * must not run concurrently on the GPU (use one stream per context).
 *
 * glint_eval_batch: frames (host array of n_frames <= 128), outs (host array
 * of n_frames device pointers, [height][width] floats each).  The first call
 * for a given batch shape (sizes, light counts, planes present) times the
 * candidate launch shapes on the context's stream, which blocks the host
 * until they finish and writes the outputs several times; later calls with
 * the same shape are asynchronous graph launches on `stream`.  Unless the
 * launch shape was set with glint_ctx_set_launch, a new batch shape re-tunes.
 * Errors: GLINT_ERR_ARG (bad counts, frames, material, or a context of
 * another device), GLINT_ERR_ALIGN, GLINT_ERR_NOT_DEVICE_PTR, GLINT_ERR_CUDA. */
typedef struct GlintContext GlintContext;
int glint_ctx_create(GlintContext** ctx);
void glint_ctx_destroy(GlintContext* ctx);
int glint_ctx_get_launch(const GlintContext* ctx, GlintLaunch* launch);
int glint_ctx_set_launch(GlintContext* ctx, const GlintLaunch* launch);
int glint_eval_batch(GlintContext* ctx, const GlintFrame* frames, int32_t n_frames,
                     const GlintMaterial* material, const GlintLight* lights,
                     float* const* outs, void* stream);

/* Adjoint (differentiation of the counting law, Sec. 3-6):
 *   grad[k] = sum_px grad_out[px] * d relaxed(px) / d theta_k,
 * theta = (alpha_x, alpha_y, ln_density, dir of light 0 (xyz), dir of light 1,
 * ...), 3 + 3 * n_lights floats; the direction entries of point lights are 0.
 * relaxed(px) is the image with every open gate counting
 * clamp(1 + mu + sigma z, 1, ceil n) instead of its floor; every discrete
 * choice (sub-footprints, LOD, cell, tetrahedron, lattice vertices, texels,
 * gates) is held fixed; interpolation weights are differentiated.  The
 * forward pass is recomputed per pixel (no stored per-texel state).
 *   grad_out:    device [height][width] float.
 *   grad:        device, 3 + 3 * n_lights floats (written).
 *   out_relaxed: device [height][width] float or NULL (the relaxed image).
 *   workspace:   device, >= glint_backward_workspace_size(frame) bytes,
 *                8-byte aligned; per-CTA partial sums (deterministic
 *                fixed-order reduction).
 * Requires the scalar material (frame->mat_px == NULL), else
 * GLINT_ERR_UNSUPPORTED; a small workspace gives GLINT_ERR_WORKSPACE. */
size_t glint_backward_workspace_size(const GlintFrame* frame);
int glint_backward(const GlintFrame* frame, const GlintMaterial* material, const GlintLight* lights,
                   const float* grad_out, float* grad, float* out_relaxed,
                   void* workspace, size_t workspace_bytes, void* stream);

/* One pass of an L2 image fit: the image, the loss and its gradient, without
 * a separate forward launch.  Per pixel the kernel evaluates the image value
 * out[px] (integer counts, as glint_eval; equal to glint_eval's image up to
 * the order of the floating-point sum, ~1e-7 relative), the relaxed value
 * and its derivatives, and weights the derivatives by 2 (out[px] -
 * target[px]): the loss of an L2 fit depends on each pixel's own value only,
 * so grad_out of glint_backward is known inside the pixel.
 *   grad[k] = sum_px 2 (out[px] - target[px]) d relaxed(px) / d theta_k
 *   *loss   = sum_px (out[px] - target[px])^2      (double-float / FP64 sums, deterministic)
 * The paper fits nothing: this entry point serves the differentiable use of
 * the model (material and light fitting against a target image).
 *   target: device [height][width] float.   out: device [height][width] float.
 *   grad:   device, 3 + 3 * n_lights floats.  loss: device float or NULL.
 *   workspace: as glint_backward.
 * Requires the scalar material (frame->mat_px == NULL), else
 * GLINT_ERR_UNSUPPORTED; a small workspace gives GLINT_ERR_WORKSPACE. */
int glint_fit_l2(const GlintFrame* frame, const GlintMaterial* material, const GlintLight* lights,
                 const float* target, float* out, float* grad, float* loss,
                 void* workspace, size_t workspace_bytes, void* stream);

/* glint_eval_batch for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is an interface for hosts that own every
 * allocation - a renderer with a fixed memory budget, code that must not
 * synchronise the device in the middle of a frame (cudaMalloc can), or a
 * plug-in inside an application with its own allocator.  Same frames,
 * material, lights and outputs as glint_eval_batch (bit-identical images),
 * but no context, no CUDA graph, no tuning (fixed 256 threads x 4 CTAs per
 * SM) and no allocation of any kind: the persistent kernel's tile counters
 * live in a static 256-byte device array that every GPU loading the library
 * keeps until the process exits.  Batches are cut into launches of up to 128
 * frames, one counter each, so n_frames may be at most 8192; more returns
 * GLINT_ERR_WORKSPACE before anything is enqueued.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, once per device, with that device current); make
 *     that first call before any stream capture.  The address is kept for the
 *     life of the process: after cudaDeviceReset on a device this entry point
 *     must not be called on that device again.
 *   - Every call uses the same array and clears the counters it needs at the
 *     start (an asynchronous memset on `stream`).  Calls whose work overlaps
 *     on the GPU - on different streams, or from different threads - race on
 *     the counters and give wrong images: order them on one stream.
 * Errors: as glint_eval_batch, plus GLINT_ERR_WORKSPACE. */
int glint_eval_batch_noalloc(const GlintFrame* frames, int32_t n_frames,
                             const GlintMaterial* material, const GlintLight* lights,
                             float* const* outs, void* stream);

/* Synthetic G-buffers generated on the GPU: the analytic ray casts that make
 * the benchmark inputs (the paper's Sec. 7.1 scenes are Unity assets; these
 * are seeded stand-ins of the same kind).  The paper has no counterpart: the
 * glint shader reads a G-buffer that a renderer already rasterised.  One
 * thread per pixel in FP64, each output rounded once to float, matching the
 * package's seeded CPU generator (scenes.py) up to the rounding of a few
 * ulps of FP64 (different sin/atan2 implementations and summation order).
 * Layouts as GlintFrame; all output pointers device, 16-byte aligned
 * (mat_px 8-byte); asynchronous on `stream`.
 *
 * Camera: pinhole at eye with orthonormal basis (fwd, right, up) and
 * vertical half-angle atan(tan_half_fov); pixel (x, y) looks along
 * fwd + sx right + sy up, sx = ((x + 0.5) 2/W - 1) tan_half_fov W/H,
 * sy = (1 - (y + 0.5) 2/H) tan_half_fov; uv derivatives by first-order ray
 * differentials (Igehy 1999). */
#define GLINT_MAX_WAVES 32

typedef struct GlintCamera {
    double eye[3];
    double fwd[3], right[3], up[3];
    double tan_half_fov;
    int32_t width, height;
} GlintCamera;

/* Heightfield y = sum_k amp[k] sin(kx[k] x + kz[k] z + phase[k]), n_waves <=
 * GLINT_MAX_WAVES, hit by marching the slab |y| <= sum amp in n_march even
 * steps to the first sign change of y - h and bisecting that bracket
 * n_bisect times.  uv = uv_scale (x, z) wrapped to [0, uv_scale); normal and
 * tangent (direction of increasing u) of the heightfield; view direction
 * -D/|D|.  Every ray must point below the horizon and the eye must lie
 * above the slab (else GLINT_ERR_ARG).  The whole frame is written. */
typedef struct GlintHeightfield {
    int32_t n_waves, n_march, n_bisect, pad;
    double kx[GLINT_MAX_WAVES], kz[GLINT_MAX_WAVES], phase[GLINT_MAX_WAVES], amp[GLINT_MAX_WAVES];
    double uv_scale;
} GlintHeightfield;
int glint_gbuffer_heightfield(const GlintCamera* camera, const GlintHeightfield* field, float* gbuf, void* stream);

/* Sphere (center, radius; uv = sphere_uv_scale (atan2(z, x)/(2 pi) + 1/2,
 * acos(y/r)/pi), tangent along increasing azimuth) on the ground plane y = 0
 * bounded by |x|, |z| <= plane_half_extent (uv = plane_uv_scale (x, z)
 * wrapped to [0, plane_uv_wrap), tangent +x); n_lights point lights (per
 * pixel: direction to the light and E = I / d^2 into light_px); material
 * plane (alpha, 10^log10 density) by bilinear value noise over two
 * [noise_h][noise_w] device grids of doubles, one value every noise_cell
 * pixels (pixel (x, y) at ((x + 0.5)/cell, (y + 0.5)/cell) of the grid).
 * Pixels that hit nothing are 0 in every plane. */
typedef struct GlintSpherePlane {
    double center[3];
    double radius, sphere_uv_scale;
    double plane_half_extent, plane_uv_scale, plane_uv_wrap;
    int32_t n_lights, noise_cell, noise_w, noise_h;
    double light_pos[GLINT_MAX_LIGHTS][3];
    double light_I[GLINT_MAX_LIGHTS];
    const double* noise_alpha;
    const double* noise_log10_density;
} GlintSpherePlane;
int glint_gbuffer_sphere_plane(const GlintCamera* camera, const GlintSpherePlane* scene, float* gbuf,
                               float* light_px, float* mat_px, void* stream);

/* Parity trace of selected pixels: for each listed pixel, a summary and the
 * records of every binomial evaluation in the canonical order (light,
 * sub-footprint, tetrahedron vertex 0..3, simplex vertex 0..2, angular
 * texel 0..3), i.e. record index ((light*K + sub)*4 + vert)*12 + sv*4 + av.
 *   px:   device, n_px int32 flat pixel indices.
 *   pix:  device, n_px records.
 *   recs: device, n_px * rec_cap records; pixel k owns recs[k*rec_cap ...];
 *         records whose canonical index is >= rec_cap are not written; slots
 *         of lights facing away from the surface are left untouched. */
typedef struct GlintTracePix {
    int32_t status;          /* 0 shaded, 1 background, 2 invalid, 3 lattice out of range */
    int32_t K;               /* sub-footprints */
    int32_t n_rec;           /* evaluation records produced (lights facing away produce none) */
    int32_t n_can_open;      /* of those, the records whose gate can open (P>=1 > 2^-26); the image
                                kernels skip a grid vertex, and a light, whose gates cannot */
    float   A, r, phi, out;  /* flakes in footprint, ratio, orientation, radiance */
} GlintTracePix;

typedef struct GlintTraceRec {
    int32_t  light, sub, vert, sv, av;
    uint32_t grid_id;        /* (level << 16) | (ring << 8) | orientation */
    int32_t  i, j;           /* simplex lattice vertex */
    int32_t  ax, ay;         /* angular texel */
    uint32_t h0, h1;         /* hash words (gate, Gaussian) */
    int32_t  gate, c;        /* gate decision, integer count */
    float    n, P1, mu, sigma, c_cont, u, v, p;
} GlintTraceRec;

int glint_eval_trace(const GlintFrame* frame, const GlintMaterial* material,
                     const GlintLight* lights, const int32_t* px, int32_t n_px,
                     GlintTracePix* pix, GlintTraceRec* recs, int32_t rec_cap, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GLINT_H */
