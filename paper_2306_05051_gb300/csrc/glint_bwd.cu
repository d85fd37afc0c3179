// Adjoint of the glint image with respect to the material roughness
// (alpha_x, alpha_y), ln(flake density) and the direction of each
// directional light.
//
// The gradient is that of the relaxed image: an open gate contributes
// clamp(1 + mu + sigma z, 1, ceil n) instead of its floor, and every discrete
// choice (sub-footprints, LOD bracket, cell, triangle, tetrahedron, lattice
// vertices, angular texels, gates) is held fixed.  The forward pass is
// recomputed per pixel with the same setup code as the image kernels; no
// per-texel state is stored.  Within a cell the interpolation weights are
// differentiated in difference form, e.g. for the simplex weights
//   sum_j du_j X_j = (qx/2)(X1 - X0) + (qy/2)(X2 - X1)   (d q / d ln rho = q/2),
// which avoids cancelling the large +-q/2 terms.  Per-pixel terms are formed
// in FP32; each thread's sums over its pixels and the warp's shuffle tree are
// double-float (exact products, Dekker sums: ~2^-44 of the summed magnitudes,
// without the FP64 pipe, which is slow on this GPU), the warps' sums go to
// FP64 and are reduced per CTA in a fixed order into the workspace, and a
// second kernel sums the CTA partials in a fixed order: deterministic.
#include "glint_kernels.cuh"

namespace glint {

constexpr int kBwdThreads = 256;
constexpr int kMaxGrad = 3 + 3 * kMaxLights;

// Derivatives of one light's per-pixel quantities.
struct LightGrad {
    bool dir;                     // directional light: its direction is a parameter
    float fx, fy;                 // angular fractions
    float dp_da[2], dp_dd[3];     // p with respect to (alpha_x, alpha_y) and the light direction
    float dfx_dd[3], dfy_dd[3];   // angular fractions with respect to the light direction
    float ds_da[2], ds_dd[3];     // shade factor with respect to the same
};

__device__ __forceinline__ float dlambda_da(int ndf, float a) {
    if (ndf == 0) return -expf(-a * a) / (3.5449077018110318f * a * a);       // 2 sqrt(pi)
    return -0.5f / (a * a * a * sqrtf(1.0f + 1.0f / (a * a)));
}

// Lambda of w (local frame) and its derivatives with respect to (alpha_x,
// alpha_y) and to w.
__device__ __forceinline__ float lambda_grad(int ndf, float ax, float ay, const float w[3], float dl_da[2],
                                             float dl_dw[3]) {
    const float s2 = (w[0] * ax) * (w[0] * ax) + (w[1] * ay) * (w[1] * ay);
    dl_da[0] = dl_da[1] = dl_dw[0] = dl_dw[1] = dl_dw[2] = 0.0f;
    if (!(s2 > 0.0f)) return 0.0f;
    const float sq = sqrtf(s2);
    const float a = w[2] / sq;
    const float lam = smith_lambda(ndf, ax, ay, w[0], w[1], w[2]);
    const float dla = dlambda_da(ndf, a);
    dl_da[0] = dla * (-a * w[0] * w[0] * ax / s2);
    dl_da[1] = dla * (-a * w[1] * w[1] * ay / s2);
    dl_dw[0] = dla * (-a * w[0] * ax * ax / s2);
    dl_dw[1] = dla * (-a * w[1] * ay * ay / s2);
    dl_dw[2] = dla / sq;
    return lam;
}

__device__ void light_grad(const KParams& P, const FrameDesc& F, const PixelSetup& S, const LocalFrame& R, int px, int l,
                           const LightState& L, LightGrad& G) {
    const KLight kl = P.lights[l];
    G.dir = kl.kind == 1;
    float d[3];
    if (kl.kind == 0) {
        const float4 lp = __ldg(F.light_px + (size_t)l * F.lstride + px);
        d[0] = lp.x; d[1] = lp.y; d[2] = lp.z;
    } else {
        d[0] = kl.dx; d[1] = kl.dy; d[2] = kl.dz;
    }
    const float dl = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const float w[3] = {d[0] / dl, d[1] / dl, d[2] / dl};
    float Fr[3][3];
    for (int c = 0; c < 3; ++c) { Fr[0][c] = R[kFrT + 2 * c]; Fr[1][c] = R[kFrB + 2 * c]; Fr[2][c] = R[kFrN + 2 * c]; }
    float ll[3], v[3];
    for (int r = 0; r < 3; ++r) { ll[r] = Fr[r][0] * w[0] + Fr[r][1] * w[1] + Fr[r][2] * w[2]; v[r] = R[kFrV + 2 * r]; }
    float hs[3] = {v[0] + ll[0], v[1] + ll[1], v[2] + ll[2]};
    const float hl = sqrtf(hs[0] * hs[0] + hs[1] * hs[1] + hs[2] * hs[2]);
    const float h[3] = {hs[0] / hl, hs[1] / hl, hs[2] / hl};
    // local light direction and half-vector with respect to the world direction d
    float Jl[3][3], Jh[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Jl[r][c] = (Fr[r][c] - ll[r] * w[c]) / dl;
    for (int c = 0; c < 3; ++c) {
        const float hj = h[0] * Jl[0][c] + h[1] * Jl[1][c] + h[2] * Jl[2][c];
        for (int r = 0; r < 3; ++r) Jh[r][c] = (Jl[r][c] - h[r] * hj) / hl;
    }
    const float ax = R[kFrAx], ay = R[kFrAy], ht = h[0], hb = h[1], hn = h[2];
    // Eq. 4: p = R D(h)/D(n)
    const float e = (ht / ax) * (ht / ax) + (hb / ay) * (hb / ay);
    float dr_dh[3], dr_da[2];
    if (P.ndf == 0) {
        const float hn2 = hn * hn;
        const float rat = expf(-e / hn2) / (hn2 * hn2);
        dr_dh[0] = rat * (-2.0f * ht / (ax * ax * hn2));
        dr_dh[1] = rat * (-2.0f * hb / (ay * ay * hn2));
        dr_dh[2] = rat * (2.0f * e / (hn2 * hn) - 4.0f / hn);
        dr_da[0] = rat * (2.0f * ht * ht / (ax * ax * ax * hn2));
        dr_da[1] = rat * (2.0f * hb * hb / (ay * ay * ay * hn2));
    } else {
        const float Dd = e + hn * hn;
        const float k = -2.0f / (Dd * Dd * Dd);
        dr_dh[0] = k * 2.0f * ht / (ax * ax);
        dr_dh[1] = k * 2.0f * hb / (ay * ay);
        dr_dh[2] = k * 2.0f * hn;
        dr_da[0] = k * (-2.0f * ht * ht / (ax * ax * ax));
        dr_da[1] = k * (-2.0f * hb * hb / (ay * ay * ay));
    }
    const bool clamped = !(L.p < 1.0f);
    for (int c = 0; c < 2; ++c) G.dp_da[c] = clamped ? 0.0f : P.R * dr_da[c];
    for (int c = 0; c < 3; ++c)
        G.dp_dd[c] = clamped ? 0.0f : P.R * (dr_dh[0] * Jh[0][c] + dr_dh[1] * Jh[1][c] + dr_dh[2] * Jh[2][c]);
    // Eq. 14: angular fractions
    const float ig = 1.0f / P.gamma;
    const float afx = ht * ig, afy = hb * ig;
    G.fx = L.v[1] + L.v[3];          // = fx (v1 + v3 = fx (1 - fy) + fx fy)
    G.fy = L.v[2] + L.v[3];
    (void)afx; (void)afy;
    for (int c = 0; c < 3; ++c) { G.dfx_dd[c] = Jh[0][c] * ig; G.dfy_dd[c] = Jh[1][c] * ig; }
    // shade = F G D(n) E / (4 R cos_v)
    const float vh = v[0] * h[0] + v[1] * h[1] + v[2] * h[2];
    const float om = 1.0f - vh;
    const float Fr_ = P.F0 + (1.0f - P.F0) * (om * om) * (om * om) * om;
    const float dF_dvh = -5.0f * (1.0f - P.F0) * (om * om) * (om * om);
    float dlv_da[2], dlv_dw[3], dll_da[2], dll_dw[3];
    const float lam_v = lambda_grad(P.ndf, ax, ay, v, dlv_da, dlv_dw);
    const float lam_l = lambda_grad(P.ndf, ax, ay, ll, dll_da, dll_dw);
    const float Gs = 1.0f / ((1.0f + lam_v) * (1.0f + lam_l));
    const float Dn = 1.0f / (3.14159265358979f * ax * ay);
    float E;
    if (kl.kind == 0) E = __ldg(F.light_px + (size_t)l * F.lstride + px).w; else E = kl.E;
    const float base = Dn * E / (4.0f * P.R * R[kFrCosV]);
    for (int c = 0; c < 2; ++c) {
        const float dG = -Gs * (dlv_da[c] / (1.0f + lam_v) + dll_da[c] / (1.0f + lam_l));
        const float dDn = -Dn / (c == 0 ? ax : ay);
        G.ds_da[c] = Fr_ * (dG * Dn + Gs * dDn) * E / (4.0f * P.R * R[kFrCosV]);
    }
    for (int c = 0; c < 3; ++c) {
        const float dvh = v[0] * Jh[0][c] + v[1] * Jh[1][c] + v[2] * Jh[2][c];
        const float dlam = dll_dw[0] * Jl[0][c] + dll_dw[1] * Jl[1][c] + dll_dw[2] * Jl[2][c];
        const float dG = -Gs * dlam / (1.0f + lam_l);
        G.ds_dd[c] = (dF_dvh * dvh * Gs + Fr_ * dG) * base;
    }
}

// One pixel: returns the relaxed radiance, writes d(relaxed)/d(theta) to
// g[0..ng) (FP32) and the radiance with integer counts (the image's value)
// to *disc.
__device__ float pixel_grad(const KParams& P, const Tables& T, const FrameDesc& F, int px, float* g, int ng,
                            float* disc) {
    for (int k = 0; k < ng; ++k) g[k] = 0.0f;
    *disc = 0.0f;
    PixelSetup S;
    LocalFrame R;
    setup_pixel<true>(P, T, F, px, S, R);
    if (S.status != 0) return 0.0f;
    float out = 0.0f, outd = 0.0f;
    float gm[3] = {0.0f, 0.0f, 0.0f};         // alpha_x, alpha_y, ln density
    // the largest trial count of the tetrahedron (P>=1 grows with N)
    const float n_max = fmaxf(fmaxf(S.ntr[0], S.ntr[1]), fmaxf(S.ntr[2], S.ntr[3]));
    for (int l = 0; l < F.nL; ++l) {
        LightState L;
        setup_light<false>(P, T, F, S, R, px, l, L);       // no angular texel record needed
        if (!L.on) continue;
        // no gate can open (P>=1 <= 2^-26 at the largest count): the light adds
        // nothing to the relaxed image or to any derivative
        if (L.p < 1.0f && -expm1f(n_max * L.lq) <= 1.4901161193847656e-8f) continue;
        LightGrad LG;
        light_grad(P, F, S, R, px, l, L, LG);
        float C = 0.0f, Cd = 0.0f, Su = 0.0f, Svx = 0.0f, Svy = 0.0f;
        float dC[3] = {0.0f, 0.0f, 0.0f}, dCd[3] = {0.0f, 0.0f, 0.0f};
        const float p = L.p;
        for (int sub = 0; sub < S.K; ++sub) {
            SubState U;
            // the sub-footprints are the same for every light, so a
            // coordinate out of range shows at the first light that is on,
            // before this pixel has added anything to mine[]
            const bool ok = P.M > 0 ? setup_sub<true, false>(P, T, S, sub, U, U.S0, U.uw, 1)
                                    : setup_sub<true, true>(P, T, S, sub, U, U.S0, U.uw, 1);
            if (!ok) {
                for (int k = 0; k < ng; ++k) g[k] = 0.0f;
                return 0.0f;
            }
#pragma unroll 1
            for (int i = 0; i < 4; ++i) {
                if (!vertex_used(P.M, i)) continue;
                const CountLaw law = count_law(S.ntr[i], S.ntr_lo[i], L.p, L.p_lo, L.lq);
                if (law.Tg <= 1u) continue;              // no gate of this grid can open
                // the 12 gates of this grid vertex first, then the open ones in
                // (simplex vertex, texel) order
                unsigned om = 0u;
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        om |= gate_open(fmix32(U.S0[3 * i + j] + L.A0[k]), law.Tg) ? (1u << (4 * j + k)) : 0u;
                float X[3] = {0.0f, 0.0f, 0.0f};
                float Z0 = 0.0f, Z1 = 0.0f;      // sum of u v and u v z over open, unclamped gates
                const float u3[3] = {U.uw[3 * i], U.uw[3 * i + 1], U.uw[3 * i + 2]};
                const uint32_t s13[3] = {U.S1[3 * i], U.S1[3 * i + 1], U.S1[3 * i + 2]};
                const float fx = LG.fx, fy = LG.fy;
                while (om) {
                    const int b = __ffs(om) - 1;
                    om &= om - 1u;
                    const int j = b >> 2, k = b & 3;
                    const float vk = k == 0 ? L.v[0] : (k == 1 ? L.v[1] : (k == 2 ? L.v[2] : L.v[3]));
                    const uint32_t a1 = k == 0 ? L.A1[0] : (k == 1 ? L.A1[1] : (k == 2 ? L.A1[2] : L.A1[3]));
                    const float uj = j == 0 ? u3[0] : (j == 1 ? u3[1] : u3[2]);
                    const uint32_t s1 = j == 0 ? s13[0] : (j == 1 ? s13[1] : s13[2]);
                    const uint32_t h1 = fmix32(s1 + a1);
                    const float z = normal_of_word(h1);
                    float cc;
                    const float cint = open_count(h1, law.mu, law.mu_lo, law.sig, law.nceil, &cc);
                    const float ck = fminf(fmaxf(cc, 1.0f), law.nceil);
                    const float xk = vk * ck;
                    X[0] += j == 0 ? xk : 0.0f;
                    X[1] += j == 1 ? xk : 0.0f;
                    X[2] += j == 2 ? xk : 0.0f;
                    C += uj * xk;
                    Cd += uj * vk * cint;
                    const float axk = k == 0 ? -(1.0f - fy) : (k == 1 ? (1.0f - fy) : (k == 2 ? -fy : fy));
                    const float ayk = k == 0 ? -(1.0f - fx) : (k == 1 ? -fx : (k == 2 ? (1.0f - fx) : fx));
                    Svx += uj * axk * ck;
                    Svy += uj * ayk * ck;
                    if (cc > 1.0f && cc < law.nceil) { Z0 += uj * vk; Z1 += uj * vk * z; }
                }
                const float hx = 0.5f * U.qx[i], hy = 0.5f * U.qy[i];
                Su += U.lower[i] ? hx * (X[1] - X[0]) + hy * (X[2] - X[1]) : hy * (X[1] - X[0]) + hx * (X[2] - X[1]);
                // d C / d theta through this vertex's count parameters:
                // d mu = nm1 dp + p dnm1;  d sigma = ((1 - p) d mu - mu dp) / (2 sigma)
                if (Z0 != 0.0f || Z1 != 0.0f) {
                    const float n = S.ntr[i];
                    const float nm1 = n > 1.0f ? n - 1.0f : 0.0f;
                    const float dnm1 = n > 1.0f ? S.dntr[i] : 0.0f;
                    const float mu = law.mu, sig = law.sig;
                    const float is2 = sig > 0.0f ? 0.5f / sig : 0.0f;
                    auto term = [&](float dp, float dn) {
                        const float dmu = nm1 * dp + p * dn;
                        return dmu * Z0 + ((1.0f - p) * dmu - mu * dp) * is2 * Z1;
                    };
                    dC[0] += term(LG.dp_da[0], 0.0f);
                    dC[1] += term(LG.dp_da[1], 0.0f);
                    dC[2] += term(0.0f, dnm1);
                    if (LG.dir)
                        for (int c = 0; c < 3; ++c) dCd[c] += term(LG.dp_dd[c], 0.0f);
                }
            }
        }
        dC[2] += Su;
        // out_l = shade C / A;  d A / d ln rho = A
        const float iA = 1.0f / S.A.hi;
        const float outl = L.shade * C * iA;
        out += outl;
        outd += L.shade * Cd * iA;
        gm[0] += (LG.ds_da[0] * C + L.shade * dC[0]) * iA;
        gm[1] += (LG.ds_da[1] * C + L.shade * dC[1]) * iA;
        gm[2] += L.shade * dC[2] * iA - outl;
        if (LG.dir)
            for (int c = 0; c < 3; ++c) {
                const float dfv = Svx * LG.dfx_dd[c] + Svy * LG.dfy_dd[c];
                g[3 + 3 * l + c] = (LG.ds_dd[c] * C + L.shade * (dCd[c] + dfv)) * iA;
            }
    }
    for (int k = 0; k < 3; ++k) g[k] = gm[k];
    *disc = outd;
    return out;
}

// Gradient of sum_px grad_out[px] * relaxed(px).  With target != NULL
// (L2 fit), grad_out is 2 (image - target) of the pixel's own image value,
// which is written to out_img, and the loss sum (image - target)^2 is
// reduced as component ng.
__global__ void __launch_bounds__(kBwdThreads, 2) bwd_kernel(const __grid_constant__ KParams P, const FrameDesc F,
                                                          const float* grad_out, const float* target,
                                                          float* out_img, float* out_relaxed,
                                                          double* partial, int ng) {
    // the double-float tables are read in the parameter block (constant
    // cache): no per-CTA copy, and the L1 keeps the shared memory it would take
    const Tables& T = P.tables;
    __shared__ double red[kBwdThreads / 32][kMaxGrad + 1];
    const int nc = target ? ng + 1 : ng;          // components reduced
    df mine[kMaxGrad + 1];
    for (int k = 0; k < nc; ++k) mine[k] = mkdf(0.0f);
    const int stride = gridDim.x * blockDim.x;
    for (int px = blockIdx.x * blockDim.x + threadIdx.x; px < F.npx; px += stride) {
        float g[kMaxGrad], disc;
        const float o = pixel_grad(P, T, F, px, g, ng, &disc);
        if (out_relaxed) out_relaxed[px] = o;
        float go;
        if (target) {
            const float r = disc - target[px];
            out_img[px] = disc;
            go = 2.0f * r;
            mine[ng] = mine[ng] + two_prod(r, r);
        } else {
            go = grad_out[px];
        }
        if (go != 0.0f)
            for (int k = 0; k < ng; ++k) mine[k] = mine[k] + two_prod(go, g[k]);
    }
    // fixed-order reduction over the CTA: a shuffle tree per warp, then the
    // warps' sums in warp order
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < nc; ++k) {
        df v = mine[k];
        for (int o = 16; o > 0; o >>= 1) {
            const df u = {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
            v = v + u;
        }
        if (lane == 0) red[w][k] = (double)v.hi + (double)v.lo;
    }
    __syncthreads();
    if ((int)threadIdx.x < nc) {
        double t = 0.0;
        for (int ww = 0; ww < kBwdThreads / 32; ++ww) t += red[ww][threadIdx.x];
        partial[(size_t)blockIdx.x * nc + threadIdx.x] = t;
    }
}

// Sum over the CTA partials of nc components: warp k sums blocks lane,
// lane + 32, ... in order, then a shuffle tree; a fixed order, so
// deterministic.  Components 0..ng-1 go to grad, component ng (if nc > ng)
// to *loss.
__global__ void bwd_reduce_kernel(const double* partial, int nblocks, int nc, int ng, float* grad, float* loss) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= nc) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partial[(size_t)b * nc + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
        if (k < ng) grad[k] = (float)s;
        else if (loss) *loss = (float)s;
    }
}

// One pixel per thread up to 8 CTAs per SM, then a grid-stride loop.
int bwd_blocks(int npx) {
    const int sms = num_sms() > 0 ? num_sms() : 1;
    const int need = (npx + kBwdThreads - 1) / kBwdThreads;
    const int cap = sms * 8;
    return need < cap ? need : cap;
}

}  // namespace glint

using namespace glint;

extern "C" {

size_t glint_backward_workspace_size(const GlintFrame* frame) {
    if (!frame || frame->width <= 0 || frame->height <= 0 || frame->n_lights < 0 || frame->n_lights > GLINT_MAX_LIGHTS)
        return 0;
    const int nc = 4 + 3 * frame->n_lights;           // the gradient and the L2 loss
    return (size_t)bwd_blocks(frame->width * frame->height) * nc * sizeof(double);
}

}  // extern "C"

namespace {

// Shared by glint_backward (grad_out given) and glint_fit_l2 (target given).
int launch_backward(const GlintFrame* frame, const GlintMaterial* material, const GlintLight* lights,
                    const float* grad_out, const float* target, float* out_img, float* grad, float* loss,
                    float* out_relaxed, void* workspace, size_t ws_bytes, void* stream) {
    int rc = check_frame_shape(frame, lights);
    if (rc) return rc;
    if (frame->mat_px) return GLINT_ERR_UNSUPPORTED;            // gradients of the scalar material only
    if (!material) return GLINT_ERR_ARG;
    if (material->lod_blend || material->sampler || material->rng_table)
        return GLINT_ERR_UNSUPPORTED;                             // ablations: forward only
    KParams P;
    if ((rc = make_material_params(material, lights, frame->n_lights, &P))) return rc;
    if ((rc = check_frame_device(frame, lights))) return rc;
    if (grad_out && (rc = check_device_ptr(grad_out, 4))) return rc;
    if (target && ((rc = check_device_ptr(target, 4)) || (rc = check_device_ptr(out_img, 4)))) return rc;
    if ((rc = check_device_ptr(grad, 4))) return rc;
    if (loss && (rc = check_device_ptr(loss, 4))) return rc;
    if (out_relaxed && (rc = check_device_ptr(out_relaxed, 4))) return rc;
    const size_t need = glint_backward_workspace_size(frame);
    if (!workspace || ws_bytes < need) return GLINT_ERR_WORKSPACE;
    if ((rc = check_device_ptr(workspace, 8))) return rc;
    const FrameDesc F = make_frame_desc(frame, nullptr);
    const int ng = 3 + 3 * frame->n_lights;
    const int nc = target ? ng + 1 : ng;
    const int blocks = bwd_blocks(F.npx);
    cudaStream_t s = (cudaStream_t)stream;
    bwd_kernel<<<blocks, kBwdThreads, 0, s>>>(P, F, grad_out, target, out_img, out_relaxed,
                                              static_cast<double*>(workspace), ng);
    if ((rc = cuda_rc(cudaGetLastError()))) return rc;
    bwd_reduce_kernel<<<1, 32 * nc, 0, s>>>(static_cast<const double*>(workspace), blocks, nc, ng, grad, loss);
    return cuda_rc(cudaGetLastError());
}

}  // namespace

extern "C" {

int glint_backward(const GlintFrame* frame, const GlintMaterial* material, const GlintLight* lights,
                   const float* grad_out, float* grad, float* out_relaxed, void* workspace, size_t ws_bytes,
                   void* stream) {
    if (!grad_out) return GLINT_ERR_ARG;
    return launch_backward(frame, material, lights, grad_out, nullptr, nullptr, grad, nullptr, out_relaxed,
                           workspace, ws_bytes, stream);
}

int glint_fit_l2(const GlintFrame* frame, const GlintMaterial* material, const GlintLight* lights,
                 const float* target, float* out, float* grad, float* loss, void* workspace, size_t ws_bytes,
                 void* stream) {
    if (!target || !out) return GLINT_ERR_ARG;
    return launch_backward(frame, material, lights, nullptr, target, out, grad, loss, nullptr, workspace,
                           ws_bytes, stream);
}

}  // extern "C"
