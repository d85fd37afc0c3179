// Per-pixel glint BRDF evaluation (device code), Deliot & Belcour 2023.
//
// One pixel, in the paper's order:
//   1. shading frame from the G-buffer                          (Sec. 3)
//   2. footprint: SVD of dUV/d(x,y) -> area, ratio, orientation  (Sec. 5.1)
//   3. sub-footprints when the ratio or area leaves the grids    (Sec. 4.2 ext.)
//   4. LOD bracket with area-linear coordinate                    (Sec. 5.2, Eq. 13)
//   5. ratio/orientation cell, pentagon triangle, prism tetrahedron
//      -> 4 grids with trials w_i f^l_i                           (Fig. 5, Sec. 6.1)
//   6. per grid: anisotropic transform + simplex lattice -> 3 texels (Eq. 12, Sec. 6.2)
//   7. per light: NDF ratio p, angular texels (4), hash, gated
//      binomial counts (48 per light), interpolation of realisations
//                                                                 (Eq. 4, Eq. 14, Sec. 6.3)
//   8. D_P = D(n)/R * C / A and the microfacet BRDF              (Eq. 2-3)
// Steps 1-6 and the angular coordinate run in double-float (see
// glint_df.cuh), and so do the count's mean (N - 1) p and 1 + mu + sigma z
// (p itself where A p > 8); the gate probability, sigma, the normal quantile
// and the hashing run in FP32 and 32-bit integers.
//
// The pieces below are shared by the image kernels (warp-cooperative, see
// glint_fwd.cu) and the per-thread parity-trace kernel.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include "glint_df.cuh"

namespace glint {

constexpr int kMaxLights = 8;
constexpr int kMaxRings = 6;
constexpr int kRotEntries = (1 << (kMaxRings + 2)) - 3;   // rings 0..6

__host__ __device__ constexpr int rot_entries(int M) { return (1 << (M + 2)) - 3; }
__host__ __device__ constexpr int rot_index(int ring, int kor) { return ring == 0 ? 0 : (1 << (ring + 1)) - 3 + kor; }

// Per (ring, orientation): the 2x2 map uv -> simplex lattice coordinate,
// up to the per-level factor sqrt(rho) f^(-l/2):
//   Q = 3^(-1/4) S diag(2^(-m/2), 2^(m/2)) Rot(-phi_k),  S = I + F2 [[1,1],[1,1]],
// stored as double-float entries (q00, q01 | q10, q11).
struct RotEntry {
    float4 r0;   // q00.hi, q00.lo, q01.hi, q01.lo
    float4 r1;   // q10.hi, q10.lo, q11.hi, q11.lo
};

struct Tables {
    DfTables d;
    RotEntry rot[kRotEntries];
};

// 32-bit words of a Tables block up to the rotation entries of ring M (the
// rotation entries start at their 16-byte aligned offset, after padding)
__host__ __device__ constexpr int tables_words(int M) {
    return (int)((offsetof(Tables, rot) + (size_t)rot_entries(M) * sizeof(RotEntry)) / 4);
}

struct KLight {
    int32_t kind;
    float dx, dy, dz, E;
};

// One frame's planes (device pointers) and size.
struct FrameDesc {
    const float4* gbuf;
    const float4* light_px;
    const float2* mat_px;
    float* out;
    int32_t W, H, npx, nL;
    int32_t lstride;             // pixels between the planes of consecutive lights (npx, or more for a band)
    int32_t tile_w;              // 0: a CTA's tile is blockDim.x consecutive pixels; else a block of
                                 // tile_w x (blockDim.x / tile_w) pixels (frame_tiles chooses)
};

// Material, lights and tables, shared by every frame of a launch.
struct KParams {
    KLight lights[kMaxLights];
    int32_t ndf;
    float ax, ay;
    float2 rho, sqrt_rho;        // double-float of exp(ln_density) and its root
    float R, F0, gamma;
    int32_t L, M, f, Kmax;
    uint32_t seed;
    int32_t lod_blend;           // 0 distributed binomial (Sec. 4.2); 1 linear mix of LOD outputs (Sec. 3)
    int32_t sampler;             // 0 gated Gaussian; 1 classical Gaussian / Bernoulli loop (Sec. 6.3)
    int32_t rng_table;           // 1: uniforms from the precomputed random-number table (Sec. 6.3)
    float top;                   // f^(L-1)
    int32_t log2f;               // log2(f): 1 or 2
    Tables tables;
};

// --------------------------------------------------------------------------
// hash: pcg3d / pcg4d (Jarzynski & Olano, JCGT 2020), MurmurHash3 fmix32
// --------------------------------------------------------------------------
__device__ __forceinline__ void pcg4d(uint32_t& x, uint32_t& y, uint32_t& z, uint32_t& w) {
    x = x * 1664525u + 1013904223u; y = y * 1664525u + 1013904223u;
    z = z * 1664525u + 1013904223u; w = w * 1664525u + 1013904223u;
    x += y * w; y += z * x; z += x * y; w += y * z;
    x ^= x >> 16; y ^= y >> 16; z ^= z >> 16; w ^= w >> 16;
    x += y * w; y += z * x; z += x * y; w += y * z;
}

__device__ __forceinline__ void pcg3d(uint32_t& x, uint32_t& y, uint32_t& z) {
    x = x * 1664525u + 1013904223u; y = y * 1664525u + 1013904223u; z = z * 1664525u + 1013904223u;
    x += y * z; y += z * x; z += x * y;
    x ^= x >> 16; y ^= y >> 16; z ^= z >> 16;
    x += y * z; y += z * x; z += x * y;
}

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16; h *= 0x85EBCA6Bu;
    h ^= h >> 13; h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// Standard normal quantile of theta = ((h >> 8) + 1/2) 2^-24, computed on
// the lower half so every theta is exact in FP32: Phi^-1(1 - x) = -Phi^-1(x).
__device__ __forceinline__ float normal_of_word(uint32_t h) {
    const uint32_t k = h >> 8;
    const bool upper = k >= (1u << 23);
    const uint32_t m = upper ? ((1u << 24) - 1u - k) : k;
    const float x = __fmul_rn(__fadd_rn((float)m, 0.5f), 5.9604644775390625e-8f);   // 2^-24
    const float z = normcdfinvf(x);
    return upper ? -z : z;
}

// --------------------------------------------------------------------------
// gated Gaussian binomial (Sec. 6.3)
// --------------------------------------------------------------------------
struct CountLaw {
    uint32_t Tg;      // gate threshold: theta0 < P>=1  <=>  ((h0 >> 7) | 1) < Tg
    float P1;
    float mu, mu_lo;  // mu = (N - 1) p in double-float (mu + mu_lo)
    float sig, nceil;
};

// ceil of a normalised double-float below 2^24
__device__ __forceinline__ float dfceil(float hi, float lo) {
    const float c = ceilf(hi);
    return (c == hi && lo > 0.0f) ? c + 1.0f : c;
}

// Counts whose mean exceeds this are formed in double-float: below it the
// FP32 mean (N - 1) p is within ~1e-5 of the exact one (relative errors of N
// and p of a few 1e-7 times a mean of at most 32).
constexpr float kDfCountMean = 32.0f;

// Parameters of the gated law for N = n + n_lo trials of success probability
// p + p_lo (both double-float).  Where N p > kDfCountMean, mu = (N - 1) p is
// formed in double-float: a count of 10^4 has an FP32 spacing of 1e-3, and
// every relative error of N or p reaches the count multiplied by mu.  P>=1
// and sigma keep FP32 (their errors move the gate by ~1e-7 relative and the
// count by ~sigma 1e-7).  lq = log1pf(-p), computed once per pixel and light
// (setup_light).
__device__ __forceinline__ CountLaw count_law(float n, float n_lo, float p, float p_lo, float lq) {
    CountLaw c;
    c.P1 = 0.0f;
    if (n > 0.0f && p > 0.0f) c.P1 = p >= 1.0f ? 1.0f : -expm1f(n * lq);
    c.Tg = (uint32_t)ceilf(c.P1 * 33554432.0f);            // 2^25
    if (n * p > kDfCountMean) {
        const df mu = (df{n, n_lo} - 1.0f) * df{p, p_lo};
        c.mu = mu.hi; c.mu_lo = mu.lo;
    } else {
        c.mu = n > 1.0f ? (n - 1.0f) * p : 0.0f;
        c.mu_lo = 0.0f;
    }
    const float var = c.mu * (1.0f - p);
    c.sig = var > 0.0f ? sqrtf(var) : 0.0f;
    c.nceil = dfceil(n, n_lo);
    return c;
}

__device__ __forceinline__ bool gate_open(uint32_t h0, uint32_t Tg) { return ((h0 >> 7) | 1u) < Tg; }

// Count of an open gate: one success plus the Gaussian stand-in for
// b(N-1, p), clamped to [1, ceil N].  1 + mu + sigma z is formed in
// double-float and floored exactly; *cc receives it rounded to FP32.
__device__ __forceinline__ float open_count(uint32_t h1, float mu, float mu_lo, float sig, float nceil, float* cc) {
    const df c = (df{mu, mu_lo} + 1.0f) + sig * normal_of_word(h1);
    float fl = floorf(c.hi);
    if (c.hi == fl && c.lo < 0.0f) fl -= 1.0f;              // c.hi - fl is exact and below 1 otherwise
    *cc = c.hi;
    return fminf(fmaxf(fl, 1.0f), nceil);
}

// --------------------------------------------------------------------------
// classical binomial approximation (Sec. 6.3, the sampler the paper
// replaces; the ablation sampler = 1)
// --------------------------------------------------------------------------
constexpr int kClassicalLoopMax = 16;

struct ClassicalLaw {
    bool gauss;       // floored Gaussian (N p > 5 or N > 16), else the Bernoulli loop
    float mu, mu_lo;  // N p (Gaussian branch, double-float where large)
    float sig;        // sqrt(N p (1 - p))
    float nceil;
    int nt;           // loop: ceil N trials
    uint32_t T, T_last;   // loop: success thresholds (((w >> 7) | 1) < T  <=>  theta < p)
};

__device__ __forceinline__ ClassicalLaw classical_law(float n, float n_lo, float p, float p_lo) {
    ClassicalLaw c;
    c.nceil = dfceil(n, n_lo);
    c.nt = 0;
    c.gauss = false;
    c.mu = c.mu_lo = c.sig = 0.0f;
    c.T = c.T_last = 0u;
    if (!(n > 0.0f) || !(p > 0.0f)) return c;
    const df np = df{n, n_lo} * df{p, p_lo};
    c.gauss = dflt(mkdf(5.0f), np) || dflt(mkdf((float)kClassicalLoopMax), df{n, n_lo});
    if (c.gauss) {
        c.mu = np.hi; c.mu_lo = np.lo;
        const float var = np.hi * (1.0f - p);
        c.sig = var > 0.0f ? sqrtf(var) : 0.0f;
    } else {
        c.nt = (int)c.nceil;
        const float fr = __fadd_rn(__fsub_rn(n, floorf(n)), n_lo);      // weight of a fractional last trial
        c.T = (uint32_t)ceilf(p * 33554432.0f);                          // 2^25
        c.T_last = fr > 0.0f ? (uint32_t)ceilf(p * fr * 33554432.0f) : c.T;
    }
    return c;
}

// Count of one evaluation with words h0, h1; *cc receives the Gaussian's
// value (or the loop count plus 1/2).
__device__ __forceinline__ float classical_count(const ClassicalLaw& L, uint32_t h0, uint32_t h1, float* cc) {
    if (L.gauss) {
        const df c = df{L.mu, L.mu_lo} + L.sig * normal_of_word(h0);
        float fl = floorf(c.hi);
        if (c.hi == fl && c.lo < 0.0f) fl -= 1.0f;
        *cc = c.hi;
        return fminf(fmaxf(fl, 0.0f), L.nceil);
    }
    float c = 0.0f;
    for (int k = 1; k <= L.nt; ++k) {
        const uint32_t w = fmix32(h1 + (uint32_t)k * 0x9E3779B9u);
        c += ((w >> 7) | 1u) < (k == L.nt ? L.T_last : L.T) ? 1.0f : 0.0f;
    }
    *cc = c + 0.5f;
    return c;
}

// --------------------------------------------------------------------------
// material functions
// --------------------------------------------------------------------------
__device__ __forceinline__ float smith_lambda(int ndf, float ax, float ay, float wt, float wb, float wn) {
    const float s2 = (wt * ax) * (wt * ax) + (wb * ay) * (wb * ay);
    if (!(s2 > 0.0f)) return 0.0f;
    const float a = wn * rsqrtf(s2);
    if (ndf == 0) return -0.5f * erfcf(a) + expf(-a * a) / (3.5449077018110318f * a);   // 2 sqrt(pi)
    return 0.5f * (sqrtf(1.0f + 1.0f / (a * a)) - 1.0f);
}

// Isotropic-grid mode (M = 0: Sec. 4 with the anisotropic footprint cut into
// pieces along its major axis, no Sec. 5 rings): the tetrahedron degenerates
// to the two LODs of the isotropic grid, vertex 0 (weight 1 - s) and vertex 3
// (weight s); vertices 1 and 2 have weight 0 and are not evaluated.
__host__ __device__ __forceinline__ bool vertex_used(int M, int i) { return M > 0 || i == 0 || i == 3; }

struct Vert {           // one tetrahedron vertex (a virtual grid)
    int ring, kor, level;
};

// --------------------------------------------------------------------------
// Steps 1-5: everything about a pixel that does not depend on a light
// --------------------------------------------------------------------------
// The struct lives on the per-thread stack (setup_sub takes it by reference),
// so each stored field costs stack traffic: what the image kernels do not
// read again is stored for the trace and adjoint kernels only.
struct PixelSetup {
    int status;         // 0 shaded, 1 background, 2 invalid
    int K, Kmaj, ksub;
    df A;               // flakes in the footprint
    df ratio, phi;      // (traces only)
    float u, v;         // centre uv (exact float inputs)
    df sig0, sig1, u0x, u0y;
    uint32_t vgid[4];   // tetrahedron vertices as grid ids: level << 16 | ring << 8 | orientation
    float ntr[4];       // trials of the 4 tetrahedron vertices (per sub-footprint)
    float ntr_lo[4];    // their low words (double-float trials)
    float wmix[4];      // linear mix (lod_blend = 1): LOD weight of each vertex's count; else 1 (set
                        // for traces only: the image kernels read it only with lod_blend)
    float dntr[4];      // d ntr / d ln(density) (adjoint)
    df srho;
};

// Shading frame (n, t, b) and view direction in it, double-float (24 words),
// with the roughness, the view's cosine and Smith Lambda (4 words): written by
// setup_pixel, read by setup_light and then dead.  The store decides where the
// 28 words live: LocalFrame keeps them with the thread (trace and adjoint
// kernels); the image kernels lend them slots of shared memory that stay idle
// until the sub-footprints are set up (SharedFrame), which keeps them off the
// per-thread stack.
constexpr int kFrN = 0, kFrT = 6, kFrB = 12, kFrV = 18;    // df vectors: word 2c (hi), 2c + 1 (lo)
constexpr int kFrAx = 24, kFrAy = 25, kFrCosV = 26, kFrLamV = 27, kFrameWords = 28;

struct LocalFrame {
    float w[kFrameWords];
    __device__ __forceinline__ float& operator[](int k) { return w[k]; }
    __device__ __forceinline__ float operator[](int k) const { return w[k]; }
};

// One lane's 28 words, bank-conflict free: words 0-15 in the lane's column of
// 16 x 32 words (row stride 32), words 16-27 in a column of 12 rows of row
// stride st.
struct SharedFrame {
    float* q;
    float* s;
    int st;
    __device__ __forceinline__ float& operator[](int k) const { return k < 16 ? q[k * 32] : s[(k - 16) * st]; }
};

template <class FS>
__device__ __forceinline__ df frame_df(const FS& R, int k) { return df{R[k], R[k + 1]}; }
template <class FS>
__device__ __forceinline__ void frame_put(FS& R, int k, df x) { R[k] = x.hi; R[k + 1] = x.lo; }

// The input planes are read once per launch: streaming (evict-first) loads
// leave the L2 to the per-thread stack of the setup state.
__device__ __forceinline__ bool load_gbuf(const FrameDesc& F, int px, float4& g0, float4& g1, float4& g2, float4& g3) {
    const float4* g = F.gbuf + (size_t)px * 4;
    g0 = __ldcs(g); g1 = __ldcs(g + 1); g2 = __ldcs(g + 2); g3 = __ldcs(g + 3);
    const float gv[15] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w, g2.x, g2.y, g2.z, g2.w, g3.x, g3.y, g3.z};
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 15; ++k) finite &= isfinite(gv[k]);
    return finite;
}

// kTrace: also store what only the trace and adjoint kernels read (d ntr /
// d ln density).
template <bool kTrace, class FS>
static __device__ __forceinline__ void setup_pixel(const KParams& P, const Tables& T, const FrameDesc& F, int px,
                                                   PixelSetup& S, FS& R) {
    S.status = 2;
    S.K = 0;
    float4 g0, g1, g2, g3;
    if (!load_gbuf(F, px, g0, g1, g2, g3)) return;

    // ---- 1. shading frame (double-float: the angular texel coordinate
    //      h_t / gamma amplifies FP32 rounding of the frame ~20x) ----------
    const float nr[3] = {g1.z, g1.w, g2.x};
    if (nr[0] == 0.0f && nr[1] == 0.0f && nr[2] == 0.0f) { S.status = 1; return; }
    const float tr[3] = {g2.y, g2.z, g2.w};
    const float vr[3] = {g3.x, g3.y, g3.z};
    df n[3], tg[3], b[3], wv[3];
    {
        const df inl = dfrsqrt(two_prod(nr[0], nr[0]) + two_prod(nr[1], nr[1]) + two_prod(nr[2], nr[2]));
        n[0] = inl * nr[0]; n[1] = inl * nr[1]; n[2] = inl * nr[2];
    }
    const df tn = n[0] * tr[0] + n[1] * tr[1] + n[2] * tr[2];
    df tp[3] = {tr[0] - tn * n[0], tr[1] - tn * n[1], tr[2] - tn * n[2]};
    const df tl2 = tp[0] * tp[0] + tp[1] * tp[1] + tp[2] * tp[2];
    const df vl2 = two_prod(vr[0], vr[0]) + two_prod(vr[1], vr[1]) + two_prod(vr[2], vr[2]);
    if (!(tl2.hi > 0.0f) || !(vl2.hi > 0.0f)) return;
    {
        const df itl = dfrsqrt(tl2);
        tg[0] = tp[0] * itl; tg[1] = tp[1] * itl; tg[2] = tp[2] * itl;
    }
    b[0] = n[1] * tg[2] - n[2] * tg[1];
    b[1] = n[2] * tg[0] - n[0] * tg[2];
    b[2] = n[0] * tg[1] - n[1] * tg[0];
    {
        const df ivl = dfrsqrt(vl2);
        wv[0] = (tg[0] * vr[0] + tg[1] * vr[1] + tg[2] * vr[2]) * ivl;
        wv[1] = (b[0] * vr[0] + b[1] * vr[1] + b[2] * vr[2]) * ivl;
        wv[2] = (n[0] * vr[0] + n[1] * vr[1] + n[2] * vr[2]) * ivl;
    }
    if (dfsign(wv[2]) <= 0) return;
    const float cos_v = wv[2].hi;

    df rho = ldf(P.rho);
    S.srho = ldf(P.sqrt_rho);
    float ax = P.ax, ay = P.ay;
    if (F.mat_px) {
        const float2 mp = __ldcs(F.mat_px + px);
        ax = ay = mp.x;
        rho = mkdf(mp.y);
        S.srho = dfsqrt(rho);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        frame_put(R, kFrN + 2 * c, n[c]);
        frame_put(R, kFrT + 2 * c, tg[c]);
        frame_put(R, kFrB + 2 * c, b[c]);
        frame_put(R, kFrV + 2 * c, wv[c]);
    }
    R[kFrAx] = ax;
    R[kFrAy] = ay;
    R[kFrCosV] = cos_v;
    R[kFrLamV] = smith_lambda(P.ndf, ax, ay, wv[0].hi, wv[1].hi, cos_v);

    // ---- 2. footprint (double-float) ----------------------------------
    // J = [[a, b], [c, d]] = [[du/dx, du/dy], [dv/dx, dv/dy]], pre-scaled by
    // a power of two so its squares stay well inside FP32 range.
    float ja = g0.z, jb = g1.x, jc = g0.w, jd = g1.y;
    int je;
    frexpf(fmaxf(fmaxf(fabsf(ja), fabsf(jb)), fmaxf(fabsf(jc), fabsf(jd))), &je);
    {
        const float s = pow2f(-je);
        ja *= s; jb *= s; jc *= s; jd *= s;
    }
    const df jE = two_prod(ja, ja) + two_prod(jb, jb);
    const df jG = two_prod(jc, jc) + two_prod(jd, jd);
    const df jF = two_prod(ja, jc) + two_prod(jb, jd);
    const df det = dfabs(two_prod(ja, jd) - two_prod(jc, jb));
    const df Pft = scale2(det, 2 * je);                 // |det J| in uv^2
    S.A = Pft * rho;                                    // flakes in the footprint
    if (!(S.A.hi > 0.0f)) return;
    const df hm = scale2(jE - jG, -1);
    const df hyp = dfsqrt(hm * hm + jF * jF);
    const df s0sq = scale2(jE + jG, -1) + hyp;
    // ratio sigma0 / max(sigma1, 2^-20 sigma0): finite for line-like footprints
    const df ratio = dflt(s0sq, scale2(det, 20)) ? s0sq / det : mkdf(1048576.0f);
    df phi = scale2(dfatan2(scale2(jF, 1), jE - jG, T.d), -1);
    if (dfsign(phi) < 0) phi = phi + ldf(T.d.pi);
    if (!dflt(phi, ldf(T.d.pi))) phi = phi - ldf(T.d.pi);
    if (kTrace) { S.ratio = ratio; S.phi = phi; }
    S.u = g0.x; S.v = g0.y;

    // ---- 3. sub-footprints --------------------------------------------
    int Kmaj = 1;
    const df rq = scale2(ratio, -P.M);
    if (dfsign(rq - 1.0f) > 0) {
        df fr;
        int c = dffloor(rq, &fr);           // rq <= 2^19 (ratio capped at 2^20)
        if (dfsign(fr) > 0) c += 1;
        Kmaj = c >= P.Kmax ? P.Kmax : c;
    }
    // (for Kmaj == 1 and K == 1 the divisions and log2(Kmaj) = 0 are exact
    // no-ops and are skipped)
    const df Ap = Kmaj == 1 ? S.A : A_over(S.A, Kmaj);
    int ksub = 1;
    while (dflt(mkdf((float)(ksub * ksub) * P.top), Ap) && Kmaj * (ksub + 1) * (ksub + 1) <= P.Kmax) ++ksub;
    const int K = Kmaj * ksub * ksub;
    S.Kmaj = Kmaj; S.ksub = ksub; S.K = K;
    const df As = K == 1 ? S.A : A_over(S.A, K);
    const df lr = dflog2(ratio, T.d);
    const df rho_r = Kmaj == 1 ? lr : lr - dflog2(mkdf((float)Kmaj), T.d);
    if (K > 1) {
        // major axis u0 of the footprint (eigenvector of J J^T for sigma0^2),
        // oriented like (cos phi, sin phi) with phi in [0, pi)
        df ex, ey;
        if (dfsign(hm) >= 0) { ex = hyp + hm; ey = jF; } else { ex = jF; ey = hyp - hm; }
        if (ex.hi == 0.0f && ey.hi == 0.0f) ex = mkdf(1.0f);
        const df inv = dfrsqrt(ex * ex + ey * ey);
        S.u0x = ex * inv; S.u0y = ey * inv;
        if (dfsign(S.u0y) < 0 || (dfsign(S.u0y) == 0 && dfsign(S.u0x) < 0)) { S.u0x = -S.u0x; S.u0y = -S.u0y; }
        S.sig0 = scale2(dfsqrt(s0sq), je);
        S.sig1 = Pft / S.sig0;
    }

    // ---- 4. LOD bracket -------------------------------------------------
    int level;
    df s;
    bool pinned;
    if (dflt(As, 1.0f)) { level = 0; s = mkdf(0.0f); pinned = true; }
    else if (!dflt(As, P.top)) { level = P.L - 2; s = mkdf(1.0f); pinned = true; }
    else {
        level = 0;
        float fl = 1.0f;
        while (!dflt(As, fl * (float)P.f)) { fl *= (float)P.f; ++level; }
        const df x = scale2(As, -level * P.log2f) - 1.0f;
        s = P.f == 4 ? x * ldf(T.d.third) : x;
        pinned = false;
    }

    // ---- 5. ratio / orientation cell, triangle, tetrahedron --------------
    df rr = rho_r;
    if (dfsign(rr) < 0) rr = mkdf(0.0f);
    if (!dflt(rr, (float)P.M)) rr = mkdf((float)P.M);
    df fx_unused;
    int m = dffloor(rr, &fx_unused);
    if (P.M > 0 && m > P.M - 1) m = P.M - 1;
    const df x = rr - (float)m;
    const int nm = m == 0 ? 4 : (1 << (m + 1));
    df t;
    int a = dffloor(scale2(phi * ldf(T.d.inv_pi), m == 0 ? 2 : m + 1), &t);
    a %= nm;
    // triangle vertices (ring, orientation) and barycentrics; scalars, not
    // arrays, so nothing below is indexed at run time
    int r0, k0, r1, k1, r2, k2;
    df lam0, lam1, lam2;
    // (M = 0, isotropic grids: rr = x = 0 here, so ring 0 takes the whole
    // weight and the ring-1 vertices get weight 0; they are not evaluated)
    if (m == 0) {
        r0 = 0; k0 = 0; r1 = 1; k1 = a; r2 = 1; k2 = (a + 1) & 3;
        lam0 = 1.0f - x;
        lam1 = x * (1.0f - t);
        lam2 = x * t;
    } else {
        // P00 = (m, a), P01 = (m, a + 1), P10 = (m + 1, 2a), P1h = (m + 1, 2a + 1), P11 = (m + 1, 2a + 2)
        const int a01 = (a + 1) % nm, a11 = (2 * a + 2) % (2 * nm);
        const df xh = scale2(x, -1);
        if (dfle(t, xh)) {                                 // P00, P10, P1h
            r0 = m; k0 = a; r1 = m + 1; k1 = 2 * a; r2 = m + 1; k2 = 2 * a + 1;
            lam0 = 1.0f - x; lam1 = x - scale2(t, 1); lam2 = scale2(t, 1);
        } else if (dfle(t, 1.0f - xh)) {                   // P00, P1h, P01
            r0 = m; k0 = a; r1 = m + 1; k1 = 2 * a + 1; r2 = m; k2 = a01;
            lam0 = (1.0f - t) - xh; lam1 = x; lam2 = t - xh;
        } else {                                           // P1h, P01, P11
            const df omt = 1.0f - t;
            r0 = m + 1; k0 = 2 * a + 1; r1 = m; k1 = a01; r2 = m + 1; k2 = a11;
            lam0 = scale2(omt, 1); lam1 = 1.0f - x; lam2 = x - scale2(omt, 1);
        }
    }
    // Prism split by vertex order: upper weight of vertex j = clamp(s - C_j,
    // 0, lam_j), C_0 = 0, C_1 = lam_0, C_2 = lam_0 + lam_1.  With c the
    // interval of s, tetrahedron vertex i sits on triangle vertex (c + i) mod 3,
    // on the upper LOD for i >= 3 - c; its weights are
    // (lam_c - (s - C_c), lam_{c+1}, lam_{c+2}, s - C_c).
    const df C1 = lam0, C2 = lam0 + lam1;
    const int c = dfle(s, C1) ? 0 : (dfle(s, C2) ? 1 : 2);
    const df sc = c == 0 ? s : (c == 1 ? s - C1 : s - C2);
    const df lc = c == 0 ? lam0 : (c == 1 ? lam1 : lam2);
    const df w[4] = {lc - sc, c == 0 ? lam1 : (c == 1 ? lam2 : lam0), c == 0 ? lam2 : (c == 1 ? lam0 : lam1), sc};
    // d s / d ln(density) = A_s / (f^l (f - 1)); the first tetrahedron vertex
    // loses and the last gains weight with s (every tetrahedron), the middle
    // two do not depend on s.  Pinned: n_i = w_i A_s.
    const float ds = pinned ? 0.0f : scale2(As, -level * P.log2f).hi / (float)(P.f - 1);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = (c + i) % 3;
        const int vring = k == 0 ? r0 : (k == 1 ? r1 : r2);
        const int vkor = k == 0 ? k0 : (k == 1 ? k1 : k2);
        const int vlevel = level + (i >= 3 - c ? 1 : 0);
        S.vgid[i] = ((uint32_t)vlevel << 16) | ((uint32_t)vring << 8) | (uint32_t)vkor;
        const df ni = pinned ? w[i] * As : scale2(w[i], vlevel * P.log2f);
        if (P.lod_blend) {
            // linear mix of LOD outputs (Sec. 3): each vertex counts over its
            // whole cell (f^level flakes; pinned: A_s) and its count is
            // weighted by w_i afterwards
            const df nf = pinned ? As : mkdf(pow2f(vlevel * P.log2f));
            S.ntr[i] = nf.hi;
            S.ntr_lo[i] = nf.lo;
            S.wmix[i] = __fadd_rn(w[i].hi, w[i].lo);
        } else {
            S.ntr[i] = ni.hi;
            S.ntr_lo[i] = ni.lo;
            if (kTrace) S.wmix[i] = 1.0f;
        }
        if (kTrace) {
            const float dw = i == 0 ? -ds : (i == 3 ? ds : 0.0f);
            S.dntr[i] = pinned ? ni.hi : dw * pow2f(vlevel * P.log2f);
        }
    }
    S.status = 0;
}

// --------------------------------------------------------------------------
// Step 7a: per light (independent of the sub-footprint)
// --------------------------------------------------------------------------
struct LightState {
    bool on;
    float p, shade;               // p of Eq. 4; F G D(n) E / (4 R cos_v)
    float p_lo;                   // low word of p (double-float where the counts can be large)
    float lq;                     // log(1 - p) (count laws)
    float v[4];                   // angular bilinear weights
    uint32_t A0[4], A1[4];        // angular hash words (kWords)
    int32_t ix0, iy0;             // angular texel of corner 0
    int32_t ax[4], ay[4];         // angular texels (traces)
};

// The four angular hash words of the texels (ix0 + (k & 1), iy0 + (k >> 1)).
__device__ __forceinline__ void angular_words(const KParams& P, int ix0, int iy0, uint32_t A0[4], uint32_t A1[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t hx = (uint32_t)(ix0 + (k & 1)), hy = (uint32_t)(iy0 + (k >> 1)), hz = ~P.seed;
        pcg3d(hx, hy, hz);
        A0[k] = hx; A1[k] = hy;
    }
}

// kTrace: also record the angular texels (ax, ay) for the trace and adjoint
// kernels; the image kernels skip those stores.  kWords: also store the four
// angular hash words; the image kernels form them in the evaluation loop
// from the stored texel (ix0, iy0) instead, which keeps 6 words per light off
// the per-thread stack for the same work when a pixel has one sub-footprint.
template <bool kTrace, class FS, bool kWords = true>
static __device__ __forceinline__ void setup_light(const KParams& P, const Tables& T, const FrameDesc& F,
                                                   const PixelSetup& S, const FS& R, int px, int l, LightState& L) {
    L.on = false;
    const KLight kl = P.lights[l];
    float lr[3], E;
    if (kl.kind == 0) {
        const float4 lp = __ldcs(F.light_px + (size_t)l * F.lstride + px);
        lr[0] = lp.x; lr[1] = lp.y; lr[2] = lp.z; E = lp.w;
    } else {
        lr[0] = kl.dx; lr[1] = kl.dy; lr[2] = kl.dz; E = kl.E;
    }
    const float ax = R[kFrAx], ay = R[kFrAy], cos_v = R[kFrCosV];
    const df ll2 = two_prod(lr[0], lr[0]) + two_prod(lr[1], lr[1]) + two_prod(lr[2], lr[2]);
    if (!(ll2.hi > 0.0f)) return;
    // light direction in the local frame, unit length
    df wl[3];
    {
        const df il = dfrsqrt(ll2);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int base = r == 0 ? kFrT : (r == 1 ? kFrB : kFrN);     // rows t, b, n of the frame
            wl[r] = (frame_df(R, base) * lr[0] + frame_df(R, base + 2) * lr[1] + frame_df(R, base + 4) * lr[2]) * il;
        }
    }
    if (dfsign(wl[2]) <= 0) return;
    const float cos_l = wl[2].hi;
    const df wv[3] = {frame_df(R, kFrV), frame_df(R, kFrV + 2), frame_df(R, kFrV + 4)};
    df h[3] = {wv[0] + wl[0], wv[1] + wl[1], wv[2] + wl[2]};
    {
        const df ih = dfrsqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
        h[0] = h[0] * ih; h[1] = h[1] * ih; h[2] = h[2] * ih;
    }
    const float ht = h[0].hi, hb = h[1].hi, hn = h[2].hi;
    // Eq. 4: p = R D(h) / D(n)
    const float e = (ht / ax) * (ht / ax) + (hb / ay) * (hb / ay);
    const float hn2 = hn * hn;
    const float rat = P.ndf == 0 ? expf(-e / hn2) / (hn2 * hn2) : 1.0f / ((e + hn2) * (e + hn2));
    L.p = fminf(P.R * rat, 1.0f);
    L.p_lo = 0.0f;
    // Where the counts can be large (A p > kDfCountMean: mu = (N - 1) p
    // reaches the count, and p's FP32 relative error of up to a few 1e-6
    // would move it by more than the count tolerance) p is formed again in
    // double-float from the double-float half-vector.
    if (L.p < 1.0f && S.A.hi * L.p > kDfCountMean) {
        const df tx = div_by(h[0], ax, approx_rcp(ax)), ty = div_by(h[1], ay, approx_rcp(ay));
        const df ed = tx * tx + ty * ty;
        const df hn2d = h[2] * h[2];
        df rd;
        if (P.ndf == 0) {
            rd = dfexp_neg(ed / hn2d, T.d) / (hn2d * hn2d);
        } else {
            const df dd = ed + hn2d;
            rd = 1.0f / (dd * dd);
        }
        df pd = rd * P.R;
        if (!dflt(pd, 1.0f)) pd = mkdf(1.0f);
        L.p = pd.hi; L.p_lo = pd.lo;
    }
    L.lq = log1pf(-L.p);
    // Eq. 14: bilinear angular texels of the projected half-vector; the
    // weights are formed from double-float fractions so each keeps full
    // relative precision however small it is.
    float fx, gx, fy, gy;
    const float ig = approx_rcp(P.gamma);
    const int ix = dffloor_w(div_by(h[0], P.gamma, ig), &fx, &gx);
    const int iy = dffloor_w(div_by(h[1], P.gamma, ig), &fy, &gy);
    L.v[0] = gx * gy; L.v[1] = fx * gy;
    L.v[2] = gx * fy; L.v[3] = fx * fy;
    L.ix0 = ix; L.iy0 = iy;
    if (kTrace) {
#pragma unroll
        for (int k = 0; k < 4; ++k) { L.ax[k] = ix + (k & 1); L.ay[k] = iy + (k >> 1); }
    }
    if (kWords) angular_words(P, ix, iy, L.A0, L.A1);
    // Eq. 2 with D_P = D(n)/R C/A: out_l = F G D(n) E / (4 R cos_v) * C / A
    const float vh = wv[0].hi * ht + wv[1].hi * hb + cos_v * hn;
    const float om = 1.0f - vh;
    const float Fr = P.F0 + (1.0f - P.F0) * (om * om) * (om * om) * om;
    const float lam_l = smith_lambda(P.ndf, ax, ay, wl[0].hi, wl[1].hi, cos_l);
    const float Gs = 1.0f / ((1.0f + R[kFrLamV]) * (1.0f + lam_l));
    const float Dn = 1.0f / (3.14159265358979f * ax * ay);
    L.shade = Fr * Gs * Dn * E / (4.0f * P.R * cos_v);
    L.on = true;
}

// --------------------------------------------------------------------------
// Step 6: spatial texels of one sub-footprint (12 = 4 grids x 3 simplex vertices)
// --------------------------------------------------------------------------
struct SubState {
    uint32_t S0[12], S1[12];      // spatial hash words
    float uw[12];                 // barycentric weights
    int32_t li[12], lj[12];       // lattice vertices (traces)
    uint32_t gid[4];
    float qx[4], qy[4];           // lattice coordinates (adjoint: d q / d ln(density) = q / 2)
    bool lower[4];                // simplex half: fx >= fy
};

// Returns false when a lattice coordinate leaves |q| < 2^30.  The spatial
// words S0 and weights of texel t go to s0[t * stride], uw[t * stride] (the
// image kernels keep those two in shared memory; pass U.S0, U.uw and stride 1
// to keep them in U).  kTrace: also record the lattice vertices and
// coordinates (li, lj, qx, qy, lower) for the trace and adjoint kernels.
// kIso: isotropic-grid mode (M = 0), vertices 0 and 3 only.
template <bool kTrace, bool kIso>
static __device__ __noinline__ bool setup_sub(const KParams& P, const Tables& T, const PixelSetup& S, int sub,
                                              SubState& U, uint32_t* s0, float* uwo, int stride) {
    df us = mkdf(S.u), vs = mkdf(S.v);
    if (S.K > 1) {
        // centre of sub-rectangle (ia, ib) of the sigma0 x sigma1 rectangle
        // aligned with (u0, u1 = (-u0y, u0x))
        const int ncols = S.Kmaj * S.ksub;
        const int ia = sub % ncols, ib = sub / ncols;
        const df oa = S.sig0 * div_by(mkdf((float)(2 * ia + 1 - ncols)), (float)(2 * ncols), 1.0f / (float)(2 * ncols));
        const df ob = S.sig1 * div_by(mkdf((float)(2 * ib + 1 - S.ksub)), (float)(2 * S.ksub), 1.0f / (float)(2 * S.ksub));
        us = us + (oa * S.u0x - ob * S.u0y);
        vs = vs + (oa * S.u0y + ob * S.u0x);
    }
    // Tetrahedron vertices 0 and 3 are the same ratio / orientation grid at
    // levels l and l + 1 (prism split, setup_pixel): with f = 4 the level
    // factor halves exactly, so vertex 3's lattice coordinate is vertex 0's
    // scaled by 1/2, bit for bit.
    df qx0, qy0;
#pragma unroll 1
    for (int ii = 0; ii < (kIso ? 2 : 4); ++ii) {
        const int i = kIso ? 3 * ii : ii;
        const uint32_t gid = S.vgid[i];
        if (kTrace) U.gid[i] = gid;
        const Vert V = {(int)((gid >> 8) & 255u), (int)(gid & 255u), (int)(gid >> 16)};
        df qx, qy;
        if (i == 3 && P.f == 4) {
            qx = scale2(qx0, -1);
            qy = scale2(qy0, -1);
        } else {
            const RotEntry Q = T.rot[rot_index(V.ring, V.kor)];
            df sl;
            if (P.f == 4) sl = scale2(S.srho, -V.level);
            else sl = (V.level & 1) ? scale2(S.srho * ldf(T.d.inv_sqrt2), -(V.level >> 1)) : scale2(S.srho, -(V.level >> 1));
            qx = sl * (df{Q.r0.x, Q.r0.y} * us + df{Q.r0.z, Q.r0.w} * vs);
            qy = sl * (df{Q.r1.x, Q.r1.y} * us + df{Q.r1.z, Q.r1.w} * vs);
            if (i == 0) { qx0 = qx; qy0 = qy; }
        }
        if (!(fabsf(qx.hi) < 1073741824.0f) || !(fabsf(qy.hi) < 1073741824.0f)) return false;
        df fxd, fyd;
        const int i0 = dffloor(qx, &fxd);
        const int j0 = dffloor(qy, &fyd);
        // barycentric weights, each rounded once from double-float fractions
        // (full relative precision)
        const bool lower = !dflt(fxd, fyd);
        if (kTrace) { U.qx[i] = qx.hi; U.qy[i] = qy.hi; U.lower[i] = lower; }
        const df hi = lower ? fxd : fyd, lo = lower ? fyd : fxd;     // larger / smaller fraction
        const df dd = hi - lo;
        const float w3[3] = {__fsub_rn(__fsub_rn(1.0f, hi.hi), hi.lo), __fadd_rn(dd.hi, dd.lo),
                             __fadd_rn(lo.hi, lo.lo)};
        const int li3[3] = {i0, lower ? i0 + 1 : i0, i0 + 1};
        const int lj3[3] = {j0, lower ? j0 : j0 + 1, j0 + 1};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (kTrace) { U.li[3 * i + j] = li3[j]; U.lj[3 * i + j] = lj3[j]; }
            uint32_t hx = (uint32_t)li3[j], hy = (uint32_t)lj3[j], hz = gid, hw = P.seed;
            pcg4d(hx, hy, hz, hw);
            s0[(3 * i + j) * stride] = hx;
            uwo[(3 * i + j) * stride] = w3[j];
            U.S1[3 * i + j] = hy;
        }
    }
    return true;
}

}  // namespace glint
