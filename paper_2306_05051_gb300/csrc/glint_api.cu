// C ABI of the glint library: argument validation, kernel parameters,
// double-float tables (built once on the host in double precision), launches.
#include <cmath>
#include <cstring>
#include <mutex>
#include "glint_kernels.cuh"

namespace glint {

namespace {

float2 split(double x) {
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}

// Build the tables once per process.
const Tables& host_tables() {
    static Tables T;
    static std::once_flag once;
    std::call_once(once, [] {
        std::memset(&T, 0, sizeof(T));
        for (int k = 0; k <= 64; ++k) {
            T.d.atan_t[k] = split(std::atan(k / 64.0));
            T.d.log2_t[k] = split(std::log2(1.0 + k / 64.0));
        }
        for (int j = 0; j < 64; ++j) T.d.exp2_t[j] = split(std::exp2(j / 64.0));
        T.d.pi = split(M_PI);
        T.d.half_pi = split(M_PI / 2);
        T.d.inv_pi = split(1.0 / M_PI);
        T.d.inv_ln2 = split(1.0 / std::log(2.0));
        T.d.inv_sqrt2 = split(1.0 / std::sqrt(2.0));
        T.d.third = split(1.0 / 3.0);
        T.d.ln2 = split(std::log(2.0));
        const double pre = std::pow(3.0, -0.25);
        const double F2 = 0.5 * (std::sqrt(3.0) - 1.0);
        for (int m = 0; m <= kMaxRings; ++m) {
            const int nk = m == 0 ? 1 : (1 << (m + 1));
            for (int k = 0; k < nk; ++k) {
                const double phi = m == 0 ? 0.0 : k * M_PI / (double)(1 << (m + 1));
                const double c = std::cos(phi), s = std::sin(phi);
                const double sx = std::pow(2.0, -0.5 * m), sy = std::pow(2.0, 0.5 * m);
                // diag(sx, sy) Rot(-phi)
                const double m00 = sx * c, m01 = sx * s, m10 = -sy * s, m11 = sy * c;
                // pre * S * (...)
                const double q00 = pre * ((1 + F2) * m00 + F2 * m10), q01 = pre * ((1 + F2) * m01 + F2 * m11);
                const double q10 = pre * (F2 * m00 + (1 + F2) * m10), q11 = pre * (F2 * m01 + (1 + F2) * m11);
                RotEntry& E = T.rot[rot_index(m, k)];
                const float2 a = split(q00), b = split(q01), cc = split(q10), d = split(q11);
                E.r0 = make_float4(a.x, a.y, b.x, b.y);
                E.r1 = make_float4(cc.x, cc.y, d.x, d.y);
            }
        }
    });
    return T;
}

int check_material(const GlintMaterial* m) {
    if (!m) return GLINT_ERR_ARG;
    if (m->ndf != 0 && m->ndf != 1) return GLINT_ERR_ARG;
    if (m->n_lods < 2 || m->n_lods > GLINT_MAX_LODS) return GLINT_ERR_ARG;
    if (m->n_rings < 0 || m->n_rings > GLINT_MAX_RINGS) return GLINT_ERR_ARG;
    if (m->lod_factor != 2 && m->lod_factor != 4) return GLINT_ERR_ARG;
    if (m->max_sub < 1 || m->max_sub > GLINT_MAX_SUB) return GLINT_ERR_ARG;
    if (!(m->R > 0.0f && m->R <= 1.0f) || !(m->gamma >= 1e-3f) || !std::isfinite(m->gamma)) return GLINT_ERR_ARG;
    if (!(m->alpha_x > 0.0f) || !(m->alpha_y > 0.0f) || !std::isfinite(m->alpha_x) || !std::isfinite(m->alpha_y))
        return GLINT_ERR_ARG;
    if (!std::isfinite(m->ln_density) || !std::isfinite(m->F0)) return GLINT_ERR_ARG;
    if ((m->lod_blend != 0 && m->lod_blend != 1) || (m->sampler != 0 && m->sampler != 1)) return GLINT_ERR_ARG;
    if (m->rng_table != 0 && m->rng_table != 1) return GLINT_ERR_ARG;
    // the table variant of the image kernels runs the anisotropic grids with the gated sampler
    if (m->rng_table && (m->sampler || m->n_rings == 0)) return GLINT_ERR_UNSUPPORTED;
    if (std::pow((double)m->lod_factor, m->n_lods - 1) * GLINT_MAX_SUB > 1e30) return GLINT_ERR_ARG;
    return GLINT_OK;
}

}  // namespace

int check_frame_shape(const GlintFrame* f, const GlintLight* lights) {
    if (!f || !f->gbuf) return GLINT_ERR_ARG;
    if (f->width <= 0 || f->height <= 0) return GLINT_ERR_ARG;
    if ((long long)f->width * f->height > 0x7fffffffLL / 4) return GLINT_ERR_ARG;
    if (f->n_lights < 0 || f->n_lights > GLINT_MAX_LIGHTS) return GLINT_ERR_ARG;
    if (f->n_lights > 0 && !lights) return GLINT_ERR_ARG;
    for (int l = 0; l < f->n_lights; ++l) {
        if (lights[l].kind != 0 && lights[l].kind != 1) return GLINT_ERR_ARG;
        if (lights[l].kind == 0 && !f->light_px) return GLINT_ERR_ARG;
        if (lights[l].kind == 1) {
            for (int c = 0; c < 3; ++c)
                if (!std::isfinite(lights[l].dir[c])) return GLINT_ERR_ARG;
            if (!std::isfinite(lights[l].intensity)) return GLINT_ERR_ARG;
        }
    }
    return GLINT_OK;
}

int check_device_ptr(const void* p, size_t align) {
    if (!p) return GLINT_ERR_ARG;
    if (((uintptr_t)p) % align) return GLINT_ERR_ALIGN;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return GLINT_ERR_NOT_DEVICE_PTR;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return GLINT_ERR_NOT_DEVICE_PTR;
    return GLINT_OK;
}

namespace {
std::mutex g_dev_mutex;
int g_sm_count[64];
constexpr int kDefaultThreads = 512;
constexpr int kDefaultCtasPerSm = 0;       // one CTA per tile, scheduled by the hardware

}  // namespace

int num_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(g_dev_mutex);
    if (dev < 0 || dev >= 64) return 0;
    if (!g_sm_count[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        g_sm_count[dev] = n;
    }
    return g_sm_count[dev];
}

static_assert(tables_words(kMaxRings) * 4 == sizeof(Tables), "the table copy must reach the last rotation entry");

int make_material_params(const GlintMaterial* m, const GlintLight* lights, int n_lights, KParams* P) {
    const int rc = check_material(m);
    if (rc) return rc;
    if (n_lights < 0 || n_lights > GLINT_MAX_LIGHTS || (n_lights > 0 && !lights)) return GLINT_ERR_ARG;
    std::memset(P, 0, sizeof(KParams));
    for (int l = 0; l < n_lights; ++l) {
        P->lights[l].kind = lights[l].kind;
        P->lights[l].dx = lights[l].dir[0]; P->lights[l].dy = lights[l].dir[1]; P->lights[l].dz = lights[l].dir[2];
        P->lights[l].E = lights[l].intensity;
    }
    P->ndf = m->ndf; P->ax = m->alpha_x; P->ay = m->alpha_y;
    const double rho = std::exp((double)m->ln_density);
    P->rho = split(rho);
    P->sqrt_rho = split(std::sqrt(rho));
    P->R = m->R; P->F0 = m->F0; P->gamma = m->gamma;
    P->L = m->n_lods; P->M = m->n_rings; P->f = m->lod_factor; P->Kmax = m->max_sub;
    P->seed = m->seed;
    P->lod_blend = m->lod_blend;
    P->sampler = m->sampler;
    P->rng_table = m->rng_table;
    P->top = (float)std::pow((double)m->lod_factor, m->n_lods - 1);
    P->log2f = m->lod_factor == 4 ? 2 : 1;
    std::memcpy(&P->tables, &host_tables(), sizeof(Tables));
    return GLINT_OK;
}

FrameDesc make_frame_desc(const GlintFrame* f, float* out) {
    FrameDesc F;
    F.gbuf = reinterpret_cast<const float4*>(f->gbuf);
    F.light_px = reinterpret_cast<const float4*>(f->light_px);
    F.mat_px = reinterpret_cast<const float2*>(f->mat_px);
    F.out = out;
    F.W = f->width; F.H = f->height; F.npx = f->width * f->height; F.nL = f->n_lights;
    F.lstride = F.npx;
    F.tile_w = 0;
    return F;
}

// Single-frame parameters: material + frame, all host-side checks.
static int make_params(const GlintFrame* f, const GlintMaterial* m, const GlintLight* lights, float* out,
                       KParams* P, FrameDesc* F) {
    int rc = check_frame_shape(f, lights);
    if (rc) return rc;
    if ((rc = make_material_params(m, lights, f->n_lights, P))) return rc;
    *F = make_frame_desc(f, out);
    return GLINT_OK;
}

int check_frame_device(const GlintFrame* f, const GlintLight* lights) {
    int rc = check_device_ptr(f->gbuf, 16);
    if (rc) return rc;
    bool need_lp = false;
    for (int l = 0; l < f->n_lights; ++l) need_lp |= lights[l].kind == 0;
    if (need_lp && (rc = check_device_ptr(f->light_px, 16))) return rc;
    if (f->mat_px && (rc = check_device_ptr(f->mat_px, 8))) return rc;
    return GLINT_OK;
}

// ctas_per_sm == 0: one CTA per tile, so the hardware block scheduler hands
// tiles to SMs as they free up (tiles differ in cost: sky, lit surface, dense
// flakes); otherwise a persistent grid of SMs x ctas_per_sm CTAs strides over
// the tiles.
FwdLaunch make_fwd_launch(int npx, int threads, int ctas_per_sm) {
    const int need = (npx + threads - 1) / threads;
    if (ctas_per_sm == 0) return FwdLaunch{threads, need};
    const int sms = num_sms() > 0 ? num_sms() : 1;
    const int cap = sms * ctas_per_sm;
    return FwdLaunch{threads, need < cap ? need : cap};
}

FwdLaunch default_fwd_launch(int npx) { return make_fwd_launch(npx, kDefaultThreads, kDefaultCtasPerSm); }

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return GLINT_OK;
    if (e == cudaErrorNoKernelImageForDevice || e == cudaErrorInvalidDeviceFunction) return GLINT_ERR_UNSUPPORTED;
    return GLINT_ERR_CUDA;
}

}  // namespace glint

namespace glint {
namespace {

// Internal copy streams of the host-buffer path, one pair per device,
// created on first use and kept for the life of the process.
struct CopyStreams {
    cudaStream_t h2d, d2h;
};
std::mutex g_copy_mutex;
CopyStreams g_copy[64];

int copy_streams(CopyStreams** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GLINT_ERR_CUDA;
    if (dev < 0 || dev >= 64) return GLINT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_copy_mutex);
    CopyStreams& c = g_copy[dev];
    if (!c.h2d && cudaStreamCreateWithFlags(&c.h2d, cudaStreamNonBlocking) != cudaSuccess) return GLINT_ERR_CUDA;
    if (!c.d2h && cudaStreamCreateWithFlags(&c.d2h, cudaStreamNonBlocking) != cudaSuccess) return GLINT_ERR_CUDA;
    *out = &c;
    return GLINT_OK;
}

constexpr size_t kBandPixels = size_t(1) << 19;     // about 0.5 M pixels per band
constexpr int kMaxBands = 64;

// Copy in, shade and copy out a frame in bands of rows, so that the
// host->device copy of band k+1, the kernel of band k and the device->host
// copy of band k-1 overlap (copy engines in both directions and the SMs).
// The caller's stream forks to the two internal copy streams through events
// and joins them again before returning, so work queued on `s` afterwards
// sees the finished image.  F: the whole frame in the staging buffer.
int host_pipeline(const GlintFrame* hf, const KParams& P, const FrameDesc& F, float* out_host, cudaStream_t s) {
    const size_t W = (size_t)hf->width, npx = (size_t)F.npx;
    size_t rows = (kBandPixels + W - 1) / W;
    if ((hf->height + rows - 1) / rows > (size_t)kMaxBands) rows = (hf->height + kMaxBands - 1) / kMaxBands;
    const int nb = (int)((hf->height + rows - 1) / rows);
    CopyStreams* cs = nullptr;
    int rc = copy_streams(&cs);
    if (rc) return rc;
    cudaEvent_t ev[2 * kMaxBands + 2];
    int nev = 0;
    auto event = [&](cudaEvent_t* e) {
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return false;
        ev[nev++] = *e;
        return true;
    };
    auto fail = [&](int code) {
        for (int k = 0; k < nev; ++k) cudaEventDestroy(ev[k]);     // released once complete
        return code;
    };
    const char* hg = reinterpret_cast<const char*>(hf->gbuf);
    const char* hl = reinterpret_cast<const char*>(hf->light_px);
    const char* hm = reinterpret_cast<const char*>(hf->mat_px);
    char* dg = reinterpret_cast<char*>(const_cast<float4*>(F.gbuf));
    char* dl = reinterpret_cast<char*>(const_cast<float4*>(F.light_px));
    char* dm = reinterpret_cast<char*>(const_cast<float2*>(F.mat_px));
    cudaEvent_t start;
    if (!event(&start)) return fail(GLINT_ERR_CUDA);
    if (cudaEventRecord(start, s) != cudaSuccess || cudaStreamWaitEvent(cs->h2d, start, 0) != cudaSuccess ||
        cudaStreamWaitEvent(cs->d2h, start, 0) != cudaSuccess)
        return fail(GLINT_ERR_CUDA);
    for (int k = 0; k < nb; ++k) {
        const size_t r0 = (size_t)k * rows;
        const size_t r1 = r0 + rows < (size_t)hf->height ? r0 + rows : (size_t)hf->height;
        const size_t b0 = r0 * W, n = (r1 - r0) * W;
        bool ok = cudaMemcpyAsync(dg + b0 * 64, hg + b0 * 64, n * 64, cudaMemcpyHostToDevice, cs->h2d) == cudaSuccess;
        if (hl)
            for (int l = 0; l < hf->n_lights && ok; ++l)
                ok = cudaMemcpyAsync(dl + (l * npx + b0) * 16, hl + (l * npx + b0) * 16, n * 16,
                                     cudaMemcpyHostToDevice, cs->h2d) == cudaSuccess;
        if (hm && ok) ok = cudaMemcpyAsync(dm + b0 * 8, hm + b0 * 8, n * 8, cudaMemcpyHostToDevice, cs->h2d) == cudaSuccess;
        cudaEvent_t in, done;
        if (!ok || !event(&in) || !event(&done)) return fail(GLINT_ERR_CUDA);
        if (cudaEventRecord(in, cs->h2d) != cudaSuccess || cudaStreamWaitEvent(s, in, 0) != cudaSuccess)
            return fail(GLINT_ERR_CUDA);
        FrameDesc Fk = F;
        Fk.gbuf = F.gbuf + b0 * 4;
        if (F.light_px) Fk.light_px = F.light_px + b0;
        if (F.mat_px) Fk.mat_px = F.mat_px + b0;
        Fk.out = F.out + b0;
        Fk.npx = (int)n;
        Fk.H = (int)(r1 - r0);
        if ((rc = cuda_rc(launch_fwd(P, Fk, s, default_fwd_launch(Fk.npx))))) return fail(rc);
        if (cudaEventRecord(done, s) != cudaSuccess || cudaStreamWaitEvent(cs->d2h, done, 0) != cudaSuccess ||
            cudaMemcpyAsync(out_host + b0, F.out + b0, n * 4, cudaMemcpyDeviceToHost, cs->d2h) != cudaSuccess)
            return fail(GLINT_ERR_CUDA);
    }
    cudaEvent_t end;
    if (!event(&end) || cudaEventRecord(end, cs->d2h) != cudaSuccess || cudaStreamWaitEvent(s, end, 0) != cudaSuccess)
        return fail(GLINT_ERR_CUDA);
    return fail(GLINT_OK);
}

}  // namespace
}  // namespace glint

using namespace glint;

extern "C" {

const char* glint_error_string(int code) {
    switch (code) {
        case GLINT_OK: return "ok";
        case GLINT_ERR_ARG: return "invalid argument";
        case GLINT_ERR_ALIGN: return "device pointer not aligned";
        case GLINT_ERR_NOT_DEVICE_PTR: return "pointer is not device memory";
        case GLINT_ERR_CUDA: return "CUDA runtime error";
        case GLINT_ERR_UNSUPPORTED: return "unsupported device or parameter";
        case GLINT_ERR_WORKSPACE: return "workspace too small";
        default: return "unknown error";
    }
}

int glint_version(void) { return 100; }

int glint_eval_launch(const GlintFrame* frame, const GlintMaterial* material, const GlintLight* lights,
                      float* out, const GlintLaunch* launch, void* stream) {
    if (!launch) return GLINT_ERR_ARG;
    const int t = launch->threads_per_cta;
    if ((t != 128 && t != 256 && t != 512 && t != 1024) || launch->ctas_per_sm < 0 || launch->ctas_per_sm > 16)
        return GLINT_ERR_ARG;
    KParams P;
    FrameDesc F;
    int rc = make_params(frame, material, lights, out, &P, &F);
    if (rc) return rc;
    if ((rc = check_frame_device(frame, lights))) return rc;
    if ((rc = check_device_ptr(out, 4))) return rc;
    return cuda_rc(launch_fwd(P, F, (cudaStream_t)stream, make_fwd_launch(F.npx, t, launch->ctas_per_sm)));
}

int glint_eval(const GlintFrame* frame, const GlintMaterial* material, const GlintLight* lights, float* out,
               void* stream) {
    KParams P;
    FrameDesc F;
    int rc = make_params(frame, material, lights, out, &P, &F);
    if (rc) return rc;
    if ((rc = check_frame_device(frame, lights))) return rc;
    if ((rc = check_device_ptr(out, 4))) return rc;
    return cuda_rc(launch_fwd(P, F, (cudaStream_t)stream, default_fwd_launch(F.npx)));
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t glint_eval_host_staging_size(int32_t width, int32_t height, int32_t n_lights, int32_t has_light_plane,
                                    int32_t has_material_plane) {
    if (width <= 0 || height <= 0 || n_lights < 0) return 0;
    const size_t npx = (size_t)width * height;
    size_t b = align256(npx * 64);
    if (has_light_plane) b += align256(npx * 16 * (size_t)n_lights);
    if (has_material_plane) b += align256(npx * 8);
    return b + align256(npx * 4);
}

int glint_eval_host(const GlintFrame* hf, const GlintMaterial* material, const GlintLight* lights,
                    float* out_host, void* staging, size_t staging_bytes, void* stream) {
    if (!hf || !out_host || !staging) return GLINT_ERR_ARG;
    int rc = check_frame_shape(hf, lights);
    if (rc) return rc;
    const size_t need = glint_eval_host_staging_size(hf->width, hf->height, hf->n_lights, hf->light_px != nullptr,
                                                     hf->mat_px != nullptr);
    if (staging_bytes < need) return GLINT_ERR_WORKSPACE;
    if ((rc = check_device_ptr(staging, 256))) return rc;
    const size_t npx = (size_t)hf->width * hf->height;
    char* base = static_cast<char*>(staging);
    GlintFrame df_ = *hf;
    size_t off = 0;
    df_.gbuf = reinterpret_cast<const float*>(base + off);
    off += align256(npx * 64);
    if (hf->light_px) {
        df_.light_px = reinterpret_cast<const float*>(base + off);
        off += align256(npx * 16 * (size_t)hf->n_lights);
    }
    if (hf->mat_px) {
        df_.mat_px = reinterpret_cast<const float*>(base + off);
        off += align256(npx * 8);
    }
    float* dout = reinterpret_cast<float*>(base + off);
    KParams P;
    FrameDesc F;
    if ((rc = make_params(&df_, material, lights, dout, &P, &F))) return rc;
    return host_pipeline(hf, P, F, out_host, (cudaStream_t)stream);
}

int glint_eval_trace(const GlintFrame* frame, const GlintMaterial* material, const GlintLight* lights,
                     const int32_t* px, int32_t n_px, GlintTracePix* pix, GlintTraceRec* recs, int32_t rec_cap,
                     void* stream) {
    if (n_px <= 0 || rec_cap < 0) return GLINT_ERR_ARG;
    KParams P;
    FrameDesc F;
    int rc = make_params(frame, material, lights, nullptr, &P, &F);
    if (rc) return rc;
    if ((rc = check_frame_device(frame, lights))) return rc;
    if ((rc = check_device_ptr(px, 4)) || (rc = check_device_ptr(pix, 4))) return rc;
    if (rec_cap > 0 && (rc = check_device_ptr(recs, 4))) return rc;
    return cuda_rc(launch_trace(P, F, px, n_px, pix, recs, rec_cap, (cudaStream_t)stream));
}

}  // extern "C"
