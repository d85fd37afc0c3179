// Synthetic G-buffers generated on the GPU: the analytic ray casts that
// produce the benchmark inputs (a displaced plane seen through a pinhole
// camera, the Heightmap and Plane views of Sec. 7.1; a sphere on a ground
// plane with point lights and a value-noise material).  One thread per
// pixel, FP64 throughout, each output rounded once to FP32, following the
// seeded CPU generator's formulas step by step.  None of the glint method's
// arithmetic is here.
#include <cmath>
#include "glint_kernels.cuh"

namespace glint {
namespace {

struct Vec3 {
    double x, y, z;
};
__device__ __forceinline__ Vec3 operator+(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ Vec3 operator-(Vec3 a, Vec3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ Vec3 operator*(double s, Vec3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ Vec3 normalize(Vec3 a) {
    const double n = fmax(sqrt(a.x * a.x + a.y * a.y + a.z * a.z), 1e-300);
    return {a.x / n, a.y / n, a.z / n};
}
__device__ __forceinline__ Vec3 ld3(const double v[3]) { return {v[0], v[1], v[2]}; }

// Pinhole camera ray through pixel (x, y): unnormalised direction and its
// (constant) screen derivatives.
__device__ __forceinline__ void camera_ray(const GlintCamera& C, int x, int y, Vec3& D, Vec3& dDdx, Vec3& dDdy) {
    const double aspect = (double)C.width / (double)C.height;
    const double xs = ((double)x + 0.5) * (2.0 / C.width) - 1.0;
    const double ys = 1.0 - ((double)y + 0.5) * (2.0 / C.height);
    const Vec3 fwd = ld3(C.fwd), right = ld3(C.right), up = ld3(C.up);
    const double sx = xs * C.tan_half_fov * aspect, sy = ys * C.tan_half_fov;
    D = fwd + (sx * right) + (sy * up);
    dDdx = ((2.0 / C.width) * C.tan_half_fov * aspect) * right;
    dDdy = (-(2.0 / C.height) * C.tan_half_fov) * up;
}

// First-order ray differential of the hit point (Igehy 1999):
// dP = t (dD - (dD.N)/(D.N) D).
__device__ __forceinline__ Vec3 transfer(double t, Vec3 D, Vec3 dD, Vec3 N) {
    const double dn = dot(D, N);
    return t * (dD - (dot(dD, N) / dn) * D);
}

// r = a - b floor(a / b), in [0, b) for b > 0 (the remainder of floored division)
__device__ __forceinline__ double wrap(double a, double b) {
    double r = fmod(a, b);
    if (r != 0.0 && ((r < 0.0) != (b < 0.0))) r += b;
    return r;
}

__device__ __forceinline__ void store_gbuf(float* g, double u, double v, double dudx, double dvdx, double dudy,
                                           double dvdy, Vec3 n, Vec3 t, Vec3 w) {
    float4* o = reinterpret_cast<float4*>(g);
    o[0] = make_float4((float)u, (float)v, (float)dudx, (float)dvdx);
    o[1] = make_float4((float)dudy, (float)dvdy, (float)n.x, (float)n.y);
    o[2] = make_float4((float)n.z, (float)t.x, (float)t.y, (float)t.z);
    o[3] = make_float4((float)w.x, (float)w.y, (float)w.z, 0.0f);
}

// ---------------------------------------------------------------------------
// heightfield y = sum_k a_k sin(kx_k x + kz_k z + phase_k)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double hf_height(const GlintHeightfield& H, double x, double z) {
    double h = 0.0;
    for (int k = 0; k < H.n_waves; ++k) h += H.amp[k] * sin(x * H.kx[k] + z * H.kz[k] + H.phase[k]);
    return h;
}

__global__ void heightfield_kernel(const __grid_constant__ GlintCamera C, const __grid_constant__ GlintHeightfield H,
                                   float* gbuf) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= C.width * C.height) return;
    const int x = px % C.width, y = px / C.width;
    Vec3 D, dDdx, dDdy;
    camera_ray(C, x, y, D, dDdx, dDdy);
    const Vec3 eye = ld3(C.eye);
    double A = 0.0;
    for (int k = 0; k < H.n_waves; ++k) A += H.amp[k];
    // march the slab |y| <= A in even steps to the first + -> - change of
    // y - h, then bisect that bracket
    auto f = [&](double t) { return eye.y + t * D.y - hf_height(H, eye.x + t * D.x, eye.z + t * D.z); };
    const double t_in = (A - eye.y) / D.y, t_out = (-A - eye.y) / D.y;
    const double step = (t_out - t_in) / H.n_march;
    double lo = t_in, hi = t_out;
    for (int j = 1; j <= H.n_march; ++j) {
        const double tj = t_in + j * step;
        if (f(tj) <= 0.0) { lo = tj - step; hi = tj; break; }
    }
    for (int b = 0; b < H.n_bisect; ++b) {
        const double mid = 0.5 * (lo + hi);
        if (f(mid) > 0.0) lo = mid; else hi = mid;
    }
    const double t = hi;
    const Vec3 P = eye + t * D;
    double hx = 0.0, hz = 0.0;
    for (int k = 0; k < H.n_waves; ++k) {
        const double c = H.amp[k] * cos(P.x * H.kx[k] + P.z * H.kz[k] + H.phase[k]);
        hx += c * H.kx[k];
        hz += c * H.kz[k];
    }
    const Vec3 N = normalize({-hx, 1.0, -hz});
    const Vec3 dPdx = transfer(t, D, dDdx, N), dPdy = transfer(t, D, dDdy, N);
    const double s = H.uv_scale;
    const Vec3 tg = normalize({1.0, hx, 0.0});
    store_gbuf(gbuf + (size_t)px * 16, wrap(s * P.x, s), wrap(s * P.z, s), s * dPdx.x, s * dPdx.z, s * dPdy.x,
               s * dPdy.z, N, tg, normalize(-1.0 * D));
}

// ---------------------------------------------------------------------------
// sphere on a bounded ground plane, point lights, value-noise material
// ---------------------------------------------------------------------------
__device__ __forceinline__ double value_noise(const double* grid, int gw, int cell, int x, int y) {
    const double ys = ((double)y + 0.5) / cell, xs = ((double)x + 0.5) / cell;
    const int y0 = (int)floor(ys), x0 = (int)floor(xs);
    const double fy = ys - y0, fx = xs - x0;
    const double g00 = grid[y0 * gw + x0], g01 = grid[y0 * gw + x0 + 1];
    const double g10 = grid[(y0 + 1) * gw + x0], g11 = grid[(y0 + 1) * gw + x0 + 1];
    return (1 - fy) * ((1 - fx) * g00 + fx * g01) + fy * ((1 - fx) * g10 + fx * g11);
}

__global__ void sphere_plane_kernel(const __grid_constant__ GlintCamera C, const __grid_constant__ GlintSpherePlane S,
                                    float* gbuf, float* light_px, float* mat_px) {
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const int npx = C.width * C.height;
    if (px >= npx) return;
    const int x = px % C.width, y = px / C.width;
    Vec3 D, dDdx, dDdy;
    camera_ray(C, x, y, D, dDdx, dDdy);
    const Vec3 eye = ld3(C.eye), ctr = ld3(S.center);
    // sphere hit
    const Vec3 oc = eye - ctr;
    const double a = dot(D, D), b = 2.0 * dot(D, oc), c = dot(oc, oc) - S.radius * S.radius;
    const double disc = b * b - 4 * a * c;
    double ts = (-b - sqrt(fmax(disc, 0.0))) / (2 * a);
    if (!(disc > 0.0) || !(ts > 0.0)) ts = INFINITY;
    // ground plane y = 0, |x|, |z| <= half extent
    double tp = (0.0 - eye.y) / D.y;
    const Vec3 Pp = eye + tp * D;
    if (!(tp > 0.0) || !(fabs(Pp.x) <= S.plane_half_extent) || !(fabs(Pp.z) <= S.plane_half_extent)) tp = INFINITY;
    const bool sphere = ts < tp;
    const bool hit = isfinite(fmin(ts, tp));
    float* g = gbuf + (size_t)px * 16;
    if (!hit) {
        for (int k = 0; k < 16; ++k) g[k] = 0.0f;
        for (int l = 0; l < S.n_lights; ++l)
            reinterpret_cast<float4*>(light_px)[(size_t)l * npx + px] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        reinterpret_cast<float2*>(mat_px)[px] = make_float2(0.0f, 0.0f);
        return;
    }
    double u, v, dudx, dvdx, dudy, dvdy;
    Vec3 P, N, tg;
    if (sphere) {
        const double t = ts;
        P = eye + t * D;
        const Vec3 Pc = P - ctr;
        N = (1.0 / S.radius) * Pc;
        const Vec3 dPdx = transfer(t, D, dDdx, N), dPdy = transfer(t, D, dDdy, N);
        const double X = Pc.x, Y = Pc.y, Z = Pc.z;
        const double rxz2 = fmax(X * X + Z * Z, 1e-30);
        const double phi = atan2(Z, X);
        const double th = acos(fmin(fmax(Y / S.radius, -1.0), 1.0));
        u = S.sphere_uv_scale * (phi / (2 * M_PI) + 0.5);
        v = S.sphere_uv_scale * th / M_PI;
        const Vec3 gphi = {-Z / rxz2, 0.0, X / rxz2};
        const double r = sqrt(dot(Pc, Pc));
        const double sin_th = sqrt(rxz2) / r;
        const Vec3 ey = {0.0, 1.0, 0.0};
        const Vec3 q = {ey.x / r - (Y / (r * r * r)) * Pc.x, ey.y / r - (Y / (r * r * r)) * Pc.y,
                        ey.z / r - (Y / (r * r * r)) * Pc.z};
        const double st = fmax(sin_th, 1e-30);
        const Vec3 gth = {-q.x / st, -q.y / st, -q.z / st};
        const Vec3 du = (S.sphere_uv_scale / (2 * M_PI)) * gphi, dv = (S.sphere_uv_scale / M_PI) * gth;
        dudx = dot(du, dPdx); dudy = dot(du, dPdy);
        dvdx = dot(dv, dPdx); dvdy = dot(dv, dPdy);
        tg = normalize({-Z, 0.0, X});
    } else {
        const double t = tp;
        P = eye + t * D;
        N = {0.0, 1.0, 0.0};
        const Vec3 dPdx = transfer(t, D, dDdx, N), dPdy = transfer(t, D, dDdy, N);
        const double s = S.plane_uv_scale;
        u = wrap(s * P.x, S.plane_uv_wrap);
        v = wrap(s * P.z, S.plane_uv_wrap);
        dudx = s * dPdx.x; dvdx = s * dPdx.z;
        dudy = s * dPdy.x; dvdy = s * dPdy.z;
        tg = {1.0, 0.0, -0.0};                 // (cos 0, 0, -sin 0)
    }
    store_gbuf(g, u, v, dudx, dvdx, dudy, dvdy, N, tg, normalize(-1.0 * D));
    for (int l = 0; l < S.n_lights; ++l) {
        const Vec3 d = ld3(S.light_pos[l]) - P;
        const double dist2 = dot(d, d);
        const double dl = sqrt(dist2);
        reinterpret_cast<float4*>(light_px)[(size_t)l * npx + px] =
            make_float4((float)(d.x / dl), (float)(d.y / dl), (float)(d.z / dl), (float)(S.light_I[l] / dist2));
    }
    const double al = value_noise(S.noise_alpha, S.noise_w, S.noise_cell, x, y);
    const double lr = value_noise(S.noise_log10_density, S.noise_w, S.noise_cell, x, y);
    reinterpret_cast<float2*>(mat_px)[px] = make_float2((float)al, (float)pow(10.0, lr));
}

int check_camera(const GlintCamera* C) {
    if (!C || C->width <= 0 || C->height <= 0 || (long long)C->width * C->height > 0x7fffffffLL / 16)
        return GLINT_ERR_ARG;
    if (!(C->tan_half_fov > 0.0) || !std::isfinite(C->tan_half_fov)) return GLINT_ERR_ARG;
    return GLINT_OK;
}

}  // namespace
}  // namespace glint

using namespace glint;

extern "C" {

int glint_gbuffer_heightfield(const GlintCamera* camera, const GlintHeightfield* field, float* gbuf, void* stream) {
    int rc = check_camera(camera);
    if (rc) return rc;
    if (!field || field->n_waves < 0 || field->n_waves > GLINT_MAX_WAVES || field->n_march < 1 ||
        field->n_bisect < 0 || !(field->uv_scale > 0.0))
        return GLINT_ERR_ARG;
    double A = 0.0;
    for (int k = 0; k < field->n_waves; ++k) A += field->amp[k];
    // every ray must enter the slab from above and leave it below
    if (!(camera->eye[1] > A)) return GLINT_ERR_ARG;
    for (int cy = 0; cy < 2; ++cy)
        for (int cx = 0; cx < 2; ++cx) {
            const double th = camera->tan_half_fov, asp = (double)camera->width / camera->height;
            const double sx = (cx ? 1.0 : -1.0) * th * asp, sy = (cy ? 1.0 : -1.0) * th;
            if (!(camera->fwd[1] + sx * camera->right[1] + sy * camera->up[1] < 0.0)) return GLINT_ERR_ARG;
        }
    if ((rc = check_device_ptr(gbuf, 16))) return rc;
    const int npx = camera->width * camera->height;
    heightfield_kernel<<<(npx + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*camera, *field, gbuf);
    return cuda_rc(cudaGetLastError());
}

int glint_gbuffer_sphere_plane(const GlintCamera* camera, const GlintSpherePlane* scene, float* gbuf,
                               float* light_px, float* mat_px, void* stream) {
    int rc = check_camera(camera);
    if (rc) return rc;
    if (!scene || !(scene->radius > 0.0) || scene->n_lights < 0 || scene->n_lights > GLINT_MAX_LIGHTS ||
        !(scene->plane_uv_wrap > 0.0) || scene->noise_cell < 1 || !scene->noise_alpha || !scene->noise_log10_density)
        return GLINT_ERR_ARG;
    if (scene->noise_w < camera->width / scene->noise_cell + 2 || scene->noise_h < camera->height / scene->noise_cell + 2)
        return GLINT_ERR_ARG;
    if ((rc = check_device_ptr(gbuf, 16)) || (rc = check_device_ptr(mat_px, 8))) return rc;
    if (scene->n_lights > 0 && (rc = check_device_ptr(light_px, 16))) return rc;
    if ((rc = check_device_ptr(scene->noise_alpha, 8)) || (rc = check_device_ptr(scene->noise_log10_density, 8)))
        return rc;
    const int npx = camera->width * camera->height;
    sphere_plane_kernel<<<(npx + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*camera, *scene, gbuf, light_px, mat_px);
    return cuda_rc(cudaGetLastError());
}

}  // extern "C"
