/*
 * Plain FP64 CPU oracle of the glint BRDF of Deliot & Belcour, "Real-Time
 * Rendering of Glinty Appearances using Distributed Binomial Laws on
 * Anisotropic Grids" (HPG 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only users.  The CUDA library never loads,
 * calls or links it, and the two share no source, header, table or constant.
 *
 * Every function follows the paper's steps in the paper's order, in double
 * precision, one pixel at a time, with no blocking, fusion or reordering.
 * Where the paper is silent or ambiguous the reading taken is stated at the
 * function; the full list of readings is kept with the design notes.
 *
 * The arithmetic is written once as templates on the number type T:
 *   T = double : the forward evaluation (integer counts, or the relaxed
 *                counts used for finite differences);
 *   T = Dual   : value plus six tangents, giving the exact FP64 derivative of
 *                the relaxed image with respect to (alpha_x, alpha_y,
 *                ln density, light direction x, y, z).
 * Discrete decisions (floors, cell, triangle and tetrahedron choice, gates)
 * always use the value part only.
 *
 * Pins (what checks this code against something other than itself) live in
 * tests/: library routines (numpy SVD, scipy ndtri/binom), quadrature of the
 * NDF and of the Smith masking integral, the paper's Fig. 5/6 discretisation,
 * brute-force flake simulation, binomial statistics and convergence.
 * The integer hash (Step 8) is "parity unpinned": the paper draws its random
 * numbers from a precomputed texture and prints none; the hash is fixed by
 * this library's specification and only its statistics are tested.
 */
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdio>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

/* ------------------------------------------------------------------------ */
/* Forward-mode dual numbers (value + NG tangents).                          */
/* ------------------------------------------------------------------------ */
constexpr int NG = 6;

struct Dual {
    double v;
    double d[NG];
    Dual() : v(0.0) { for (int k = 0; k < NG; ++k) d[k] = 0.0; }
    Dual(double x) : v(x) { for (int k = 0; k < NG; ++k) d[k] = 0.0; }
};

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }

inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int k = 0; k < NG; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int k = 0; k < NG; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int k = 0; k < NG; ++k) r.d[k] = -a.d[k]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int k = 0; k < NG; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) { Dual r(a.v / b.v); for (int k = 0; k < NG; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v; return r; }
inline Dual operator+(const Dual& a, double b) { return a + Dual(b); }
inline Dual operator+(double a, const Dual& b) { return Dual(a) + b; }
inline Dual operator-(const Dual& a, double b) { return a - Dual(b); }
inline Dual operator-(double a, const Dual& b) { return Dual(a) - b; }
inline Dual operator*(const Dual& a, double b) { Dual r(a.v * b); for (int k = 0; k < NG; ++k) r.d[k] = a.d[k] * b; return r; }
inline Dual operator*(double a, const Dual& b) { return b * a; }
inline Dual operator/(const Dual& a, double b) { return a * (1.0 / b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }

inline double sqrt(double a) { return std::sqrt(a); }
inline double exp(double a) { return std::exp(a); }
inline double expm1(double a) { return std::expm1(a); }
inline double log1p(double a) { return std::log1p(a); }
inline double erfc(double a) { return std::erfc(a); }

inline Dual chain(const Dual& a, double f, double df) { Dual r(f); for (int k = 0; k < NG; ++k) r.d[k] = df * a.d[k]; return r; }
inline Dual sqrt(const Dual& a) { double s = std::sqrt(a.v); return chain(a, s, s > 0 ? 0.5 / s : 0.0); }
inline Dual exp(const Dual& a) { double e = std::exp(a.v); return chain(a, e, e); }
inline Dual expm1(const Dual& a) { return chain(a, std::expm1(a.v), std::exp(a.v)); }
inline Dual log1p(const Dual& a) { return chain(a, std::log1p(a.v), 1.0 / (1.0 + a.v)); }
inline Dual erfc(const Dual& a) { return chain(a, std::erfc(a.v), -2.0 / std::sqrt(M_PI) * std::exp(-a.v * a.v)); }

template <class T> inline T sq(const T& x) { return x * x; }

/* ------------------------------------------------------------------------ */
/* Public parameter blocks (mirrored by oracle/__init__.py with ctypes).     */
/* ------------------------------------------------------------------------ */
struct OMaterial {
    int32_t ndf;          /* 0 Beckmann, 1 GGX */
    float alpha_x, alpha_y;
    float ln_density;     /* ln(flakes per uv^2) when no per-pixel plane */
    float R;              /* Eq. 4 ratio */
    float F0;
    float gamma;          /* angular texel size in projected half-vector units */
    int32_t n_lods;       /* L */
    int32_t n_rings;      /* M */
    int32_t lod_factor;   /* f (2 or 4) */
    int32_t max_sub;      /* K_max */
    uint32_t seed;
    int32_t lod_blend;    /* 0 distributed binomial (Sec. 4.2); 1 linear mix of outputs (Sec. 3) */
    int32_t sampler;      /* 0 gated Gaussian (Sec. 6.3); 1 classical Gaussian / Bernoulli loop (Sec. 6.3) */
    int32_t rng_table;    /* 0 per-evaluation hash; 1 uniforms fetched from a precomputed table (Sec. 6.3) */
};

struct OLight {
    int32_t kind;         /* 0 point (direction and E from the per-pixel plane), 1 directional */
    float dir[3];
    float intensity;
};

struct OPix {              /* per-pixel summary */
    int32_t status;       /* 0 shaded, 1 background, 2 invalid, 3 lattice out of range */
    int32_t K, Kmaj, k;
    double A, r, phi, s0, s1;
    double out;
};

struct ORec {              /* one binomial evaluation (for parity traces) */
    int32_t light, sub, vert, sv, av;
    int32_t level, ring, kor, tri, tet, pinned;
    uint32_t gid;
    int32_t i, j, ax, ay;
    uint32_t h0, h1;
    int32_t gate, c;
    double n, p, P1, mu, sigma, z, c_cont, u, v;
    double x, t, s, As, qx, qy, afx, afy;
    double w;              /* tetrahedron weight of the record's grid vertex */
};

struct Scene {
    const float* gbuf;     /* [H][W][16] */
    const float* light_px; /* [nL][H][W][4] or null */
    const float* mat_px;   /* [H][W][2] (alpha, density) or null */
    int W, H, nL;
    OMaterial mat;
    const OLight* lights;
};

struct Trace {             /* optional sink for one pixel */
    OPix* pix;
    ORec* recs;
    int cap;
    int n;
};

/* ------------------------------------------------------------------------ */
/* Standard normal quantile, Phi^-1.  Definition: the z with Phi(z) = P,     */
/* Phi(z) = erfc(-z/sqrt 2)/2.  Solved by Newton's method on that            */
/* definition, started from Abramowitz & Stegun 26.2.23.                     */
/* ------------------------------------------------------------------------ */
double phi_cdf(double z) { return 0.5 * std::erfc(-z / std::sqrt(2.0)); }

double phi_inv(double P) {
    if (!(P > 0.0 && P < 1.0)) return P <= 0.0 ? -INFINITY : INFINITY;
    const bool upper = P > 0.5;
    const double q = upper ? 1.0 - P : P;           /* lower-tail probability */
    const double t = std::sqrt(-2.0 * std::log(q));
    double z = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                     (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
    for (int it = 0; it < 60; ++it) {
        const double f = phi_cdf(z) - q;
        const double dens = std::exp(-0.5 * z * z) / std::sqrt(2.0 * M_PI);
        const double step = f / dens;
        z -= step;
        if (std::fabs(step) <= 1e-16 * (1.0 + std::fabs(z))) break;
    }
    return upper ? -z : z;
}

/* ------------------------------------------------------------------------ */
/* Step 8 - integer hash.  The paper fetches its two uniforms from a         */
/* precomputed random texture (Sec. 6.3, last paragraph); this library       */
/* replaces it with a counter hash.  pcg3d / pcg4d follow Jarzynski & Olano, */
/* "Hash Functions for GPU Rendering", JCGT 9(3) 2020; fmix32 is the         */
/* MurmurHash3 finaliser (Appleby).  Parity unpinned against the paper.      */
/* ------------------------------------------------------------------------ */
void pcg4d(uint32_t v[4]) {
    for (int k = 0; k < 4; ++k) v[k] = v[k] * 1664525u + 1013904223u;
    v[0] += v[1] * v[3]; v[1] += v[2] * v[0]; v[2] += v[0] * v[1]; v[3] += v[1] * v[2];
    for (int k = 0; k < 4; ++k) v[k] ^= v[k] >> 16;
    v[0] += v[1] * v[3]; v[1] += v[2] * v[0]; v[2] += v[0] * v[1]; v[3] += v[1] * v[2];
}

void pcg3d(uint32_t v[3]) {
    for (int k = 0; k < 3; ++k) v[k] = v[k] * 1664525u + 1013904223u;
    v[0] += v[1] * v[2]; v[1] += v[2] * v[0]; v[2] += v[0] * v[1];
    for (int k = 0; k < 3; ++k) v[k] ^= v[k] >> 16;
    v[0] += v[1] * v[2]; v[1] += v[2] * v[0]; v[2] += v[0] * v[1];
}

uint32_t fmix32(uint32_t h) {
    h ^= h >> 16; h *= 0x85EBCA6Bu;
    h ^= h >> 13; h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

/* Identifier of the virtual grid (LOD level, ratio ring, orientation). */
uint32_t grid_id(int level, int ring, int kor) {
    return ((uint32_t)level << 16) | ((uint32_t)ring << 8) | (uint32_t)kor;
}

/* Two hash words of the evaluation at spatial lattice vertex (i, j) of grid
 * gid and angular texel (ax, ay). */
void eval_hash(int32_t i, int32_t j, uint32_t gid, int32_t ax, int32_t ay, uint32_t seed,
               uint32_t* h0, uint32_t* h1) {
    uint32_t s[4] = {(uint32_t)i, (uint32_t)j, gid, seed};
    pcg4d(s);
    uint32_t a[3] = {(uint32_t)ax, (uint32_t)ay, ~seed};
    pcg3d(a);
    *h0 = fmix32(s[0] + a[0]);
    *h1 = fmix32(s[1] + a[1]);
}

/* Random-number table (Sec. 6.3, last paragraph: the two uniforms of an
 * evaluation fetched from a small precomputed texture of random numbers
 * instead of being computed).  The table holds 2^16 pairs of words,
 *   R[k] = (fmix32(2k * 0x9E3779B9 + 0x632BE5AB), fmix32((2k + 1) * 0x9E3779B9 + 0x632BE5AB)),
 * and the evaluation at spatial key s (first pcg4d word of the lattice
 * vertex and grid) and angular key a (first pcg3d word of the angular texel)
 * reads entry (s + a) >> 16: the spatial and angular hashes stay, the
 * per-evaluation mixing is replaced by the fetch. */
constexpr int kRngTableBits = 16;

void table_words(uint32_t k, uint32_t* h0, uint32_t* h1) {
    *h0 = fmix32(2u * k * 0x9E3779B9u + 0x632BE5ABu);
    *h1 = fmix32((2u * k + 1u) * 0x9E3779B9u + 0x632BE5ABu);
}

void eval_table(int32_t i, int32_t j, uint32_t gid, int32_t ax, int32_t ay, uint32_t seed,
                uint32_t* h0, uint32_t* h1) {
    uint32_t s[4] = {(uint32_t)i, (uint32_t)j, gid, seed};
    pcg4d(s);
    uint32_t a[3] = {(uint32_t)ax, (uint32_t)ay, ~seed};
    pcg3d(a);
    table_words((s[0] + a[0]) >> (32 - kRngTableBits), h0, h1);
}

/* Uniform in (0, 1) from the top 24 bits of a hash word. */
double theta_of(uint32_t h) { return ((double)(h >> 8) + 0.5) * 0x1p-24; }

/* ------------------------------------------------------------------------ */
/* Step 2 - NDF.  Eq. 2-4 use a standard NDF D(h) (Beckmann or GGX,         */
/* Sec. 3 and Sec. 7 "any NDF"); the anisotropic forms of Walter et al.     */
/* 2007 are written in the local frame (t, b, n).                            */
/* ------------------------------------------------------------------------ */
template <class T>
T ndf_D(int ndf, const T& ax, const T& ay, const T& ht, const T& hb, const T& hn) {
    const T e = sq(ht) / sq(ax) + sq(hb) / sq(ay);
    if (ndf == 0) return exp(-e / sq(hn)) / (M_PI * ax * ay * sq(sq(hn)));
    return 1.0 / (M_PI * ax * ay * sq(e + sq(hn)));
}

/* D(n): the NDF at the shading normal (h = n). */
template <class T>
T ndf_Dn(const T& ax, const T& ay) { return 1.0 / (M_PI * ax * ay); }

/* Smith Lambda of the same NDF (separable masking, Walter et al. 2007). */
template <class T>
T smith_lambda(int ndf, const T& ax, const T& ay, const T& wt, const T& wb, const T& wn) {
    const T s2 = sq(wt * ax) + sq(wb * ay);
    if (val(s2) <= 0.0) return T(0.0);
    const T a = wn / sqrt(s2);
    if (ndf == 0) return -0.5 * erfc(a) + exp(-sq(a)) / (2.0 * std::sqrt(M_PI) * a);
    return 0.5 * (sqrt(1.0 + 1.0 / sq(a)) - 1.0);
}

/* ------------------------------------------------------------------------ */
/* Step 3 - pixel footprint (Sec. 5.1): singular value decomposition of the  */
/* 2x2 Jacobian J = [dUV/dx | dUV/dy].  Major axis v0 = sigma0 * u0,         */
/* rotation phi = angle of u0 (reading: atan2(y, x), taken modulo pi),       */
/* ratio r = |v0| / |v1|, footprint area P = sigma0 * sigma1 = |det J|.      */
/* ------------------------------------------------------------------------ */
struct Footprint { double s0, s1, phi, P, r; };

Footprint footprint(double a, double b, double c, double d) {
    /* J = [[a, b], [c, d]]; its left singular vectors are the eigenvectors
     * of J J^T = [[E, F], [F, G]]. */
    const double E = a * a + b * b, G = c * c + d * d, F = a * c + b * d;
    const double det = a * d - b * c;
    Footprint fp;
    fp.P = std::fabs(det);
    const double h = std::hypot(0.5 * (E - G), F);
    const double s0sq = 0.5 * (E + G) + h;
    fp.s0 = std::sqrt(s0sq);
    fp.s1 = fp.s0 > 0.0 ? fp.P / fp.s0 : 0.0;
    double phi = 0.5 * std::atan2(2.0 * F, E - G);
    if (phi < 0.0) phi += M_PI;
    if (phi >= M_PI) phi -= M_PI;
    fp.phi = phi;
    /* ratio sigma0 / max(sigma1, 2^-20 sigma0): a line-like footprint keeps a
     * finite ratio (beyond 2^20 nothing changes: the sub-footprint count is
     * capped and the ring coordinate clamped at M). */
    fp.r = (fp.P > 0.0 && s0sq < 0x1p20 * fp.P) ? s0sq / fp.P : 0x1p20;
    return fp;
}

/* ------------------------------------------------------------------------ */
/* Step 4 - sub-footprints.  Not in the paper: its grids are finite (M ratio */
/* rings, L levels), and Sec. 4.2 notes that the distributed law may be     */
/* spread over more than two areas.  A footprint of ratio above 2^M is cut  */
/* along its major axis into Kmaj pieces; a piece whose area is above the   */
/* top level is cut into k x k more.  K = Kmaj k^2 <= K_max.                 */
/* ------------------------------------------------------------------------ */
struct Split { int Kmaj, k, K; };

Split split_footprint(double r, double A, int M, int L, int f, int Kmax) {
    Split s;
    const double rmax = std::ldexp(1.0, M);
    s.Kmaj = 1;
    if (r > rmax) {
        const double q = std::ceil(r / rmax);
        s.Kmaj = q >= (double)Kmax ? Kmax : (int)q;
    }
    const double Ap = A / s.Kmaj;
    const double top = std::pow((double)f, L - 1);
    s.k = 1;
    while ((double)s.k * s.k * top < Ap && s.Kmaj * (s.k + 1) * (s.k + 1) <= Kmax) ++s.k;
    s.K = s.Kmaj * s.k * s.k;
    return s;
}

/* ------------------------------------------------------------------------ */
/* Step 5 - LOD bracket (Sec. 5.2, Eq. 13 generalised to area factor f).     */
/* Level l holds f^l flakes per cell (one flake per level-0 texel, Sec. 4.1  */
/* stratified).  The s coordinate is area-linear so that the distributed     */
/* law of Sec. 4.2 (weights (P - P_lo)/(P_hi - P_lo)) holds.  Outside        */
/* [1, f^(L-1)] the coordinate is pinned to the end level and the trials are */
/* scaled to the footprint's own area.                                       */
/* ------------------------------------------------------------------------ */
template <class T> struct Lod { int level; T s; bool pinned; };

template <class T>
Lod<T> lod_bracket(const T& As, int f, int L) {
    Lod<T> r;
    const double top = std::pow((double)f, L - 1);
    if (val(As) < 1.0) { r.level = 0; r.s = T(0.0); r.pinned = true; return r; }
    if (val(As) >= top) { r.level = L - 2; r.s = T(1.0); r.pinned = true; return r; }
    int l = 0;
    double fl = 1.0;
    while (fl * f <= val(As)) { fl *= f; ++l; }
    r.level = l;
    r.s = (As - fl) / (fl * f - fl);
    r.pinned = false;
    return r;
}

/* ------------------------------------------------------------------------ */
/* Step 6 - ratio / orientation lattice (Sec. 5.2 and Fig. 5; Sec. 6.1 and  */
/* Fig. 6).  Ring m sits at ratio 2^m (radial coordinate log2 r); ring 0 is */
/* the single isotropic grid; ring m >= 1 has 2^(m+1) orientations          */
/* k pi / 2^(m+1) over [0, pi) - Fig. 5 draws the 45 degree line from ring  */
/* 1, the 22.5/67.5 lines from ring 2 and the 11.25 multiples from ring 3.  */
/* A cell between rings m and m+1 is a pentagon (two ring-m orientations,   */
/* three ring-(m+1) ones) cut into the three triangles of Fig. 6; the inner */
/* cell is a triangle fan around the isotropic apex.  Barycentrics are taken */
/* in the (log2 r, phi) parameter plane.                                     */
/* ------------------------------------------------------------------------ */
struct GridVert { int ring, kor; };
struct Cell { GridVert v[3]; double lam[3]; int tri; int m; double x, t; };

Cell ratio_cell(double rho_r, double phi, int M) {
    Cell c;
    if (M == 0) {
        /* Isotropic grids only (Sec. 4 without Sec. 5): the single grid of
         * ring 0 carries the whole weight; the footprint's anisotropy was
         * handled by the split into pieces along the major axis. */
        c.m = 0; c.x = 0.0; c.t = 0.0; c.tri = 0;
        for (int k = 0; k < 3; ++k) c.v[k] = {0, 0};
        c.lam[0] = 1.0; c.lam[1] = 0.0; c.lam[2] = 0.0;
        return c;
    }
    const double rr = std::min(std::max(rho_r, 0.0), (double)M);
    const int m = std::min((int)std::floor(rr), M - 1);
    const double x = rr - m;
    c.m = m;
    c.x = x;
    if (m == 0) {
        const double q = phi / (M_PI / 4.0);
        int a = (int)std::floor(q);
        const double t = q - a;
        a %= 4;
        c.t = t;
        c.tri = 0;
        c.v[0] = {0, 0}; c.v[1] = {1, a}; c.v[2] = {1, (a + 1) % 4};
        c.lam[0] = 1.0 - x; c.lam[1] = x * (1.0 - t); c.lam[2] = x * t;
        return c;
    }
    const int nm = 1 << (m + 1);
    const double q = phi / (M_PI / nm);
    int a = (int)std::floor(q);
    const double t = q - a;
    a %= nm;
    c.t = t;
    const GridVert P00 = {m, a}, P01 = {m, (a + 1) % nm};
    const GridVert P10 = {m + 1, 2 * a}, P1h = {m + 1, 2 * a + 1}, P11 = {m + 1, (2 * a + 2) % (2 * nm)};
    if (t <= 0.5 * x) {                       /* T1 = {(0,0), (1,0), (1,1/2)} */
        c.tri = 1;
        c.v[0] = P00; c.v[1] = P10; c.v[2] = P1h;
        c.lam[0] = 1.0 - x; c.lam[1] = x - 2.0 * t; c.lam[2] = 2.0 * t;
    } else if (t <= 1.0 - 0.5 * x) {          /* T2 = {(0,0), (1,1/2), (0,1)} */
        c.tri = 2;
        c.v[0] = P00; c.v[1] = P1h; c.v[2] = P01;
        c.lam[0] = 1.0 - t - 0.5 * x; c.lam[1] = x; c.lam[2] = t - 0.5 * x;
    } else {                                  /* T3 = {(1,1/2), (0,1), (1,1)} */
        c.tri = 3;
        c.v[0] = P1h; c.v[1] = P01; c.v[2] = P11;
        c.lam[0] = 2.0 * (1.0 - t); c.lam[1] = 1.0 - x; c.lam[2] = x - 2.0 * (1.0 - t);
    }
    return c;
}

/* Prism (triangle x [level l, level l+1]) cut into three tetrahedra by the
 * vertex order (Sec. 6.1, "each triangle becomes a prism that we can further
 * split into three tetrahedra").  Upper weight of triangle vertex j is
 * clamp(s - (lam_0 + ... + lam_{j-1}), 0, lam_j); lower weight is the rest.
 * Output: the tetrahedron's four vertices (upper flag, triangle index) and
 * barycentric weights.  Ties go to the lower-indexed tetrahedron. */
template <class T> struct TetVert { int upper; int tv; T w; };

template <class T>
int tet_split(const double lam[3], const T& s, TetVert<T> out[4]) {
    const double C1 = lam[0], C2 = lam[0] + lam[1];
    if (val(s) <= C1) {
        out[0] = {0, 0, lam[0] - s};
        out[1] = {0, 1, T(lam[1])};
        out[2] = {0, 2, T(lam[2])};
        out[3] = {1, 0, s};
        return 1;
    }
    if (val(s) <= C2) {
        out[0] = {0, 1, lam[1] - (s - C1)};
        out[1] = {0, 2, T(lam[2])};
        out[2] = {1, 0, T(lam[0])};
        out[3] = {1, 1, s - C1};
        return 2;
    }
    out[0] = {0, 2, lam[2] - (s - C2)};
    out[1] = {1, 0, T(lam[0])};
    out[2] = {1, 1, T(lam[1])};
    out[3] = {1, 2, s - C2};
    return 3;
}

/* ------------------------------------------------------------------------ */
/* Step 7 - anisotropic grid transform (Sec. 5.1, Eq. 12) and simplex       */
/* lattice (Sec. 6.2, Perlin's simplex skew).  Reading of Eq. 12: grid       */
/* (l, m, k) has cells of area a_l = f^l / rho, ratio r_m = 2^m, long side   */
/* along phi_k:  g = diag((a_l r_m)^-1/2, (r_m / a_l)^1/2) Rot(-phi_k) uv.   */
/* g is scaled by 3^-1/4 so each simplex lattice vertex owns unit area, then */
/* skewed by F2 = (sqrt 3 - 1)/2.                                            */
/* ------------------------------------------------------------------------ */
template <class T>
void grid_coords(double u, double v, int level, int ring, int kor, const T& rho, int f, T* qx, T* qy) {
    const double phik = ring == 0 ? 0.0 : kor * M_PI / (double)(1 << (ring + 1));
    const double c = std::cos(phik), s = std::sin(phik);
    const double xr = c * u + s * v;
    const double yr = -s * u + c * v;
    const double rm = std::ldexp(1.0, ring);
    const T al = std::pow((double)f, level) / rho;
    const T gx = xr / sqrt(al * rm);
    const T gy = yr * sqrt(rm / al);
    const double pre = std::pow(3.0, -0.25);
    const double F2 = 0.5 * (std::sqrt(3.0) - 1.0);
    const T hx = pre * gx, hy = pre * gy;
    const T skew = F2 * (hx + hy);
    *qx = hx + skew;
    *qy = hy + skew;
}

template <class T> struct SimplexVert { int32_t i, j; T u; };

/* The three lattice vertices of the simplex containing q, with barycentric
 * weights (Sec. 6.2: 3 evaluations with barycentric interpolation). */
template <class T>
void simplex_vertices(const T& qx, const T& qy, SimplexVert<T> out[3]) {
    const double i0 = std::floor(val(qx)), j0 = std::floor(val(qy));
    const T fx = qx - i0, fy = qy - j0;
    const int32_t I = (int32_t)i0, J = (int32_t)j0;
    if (val(fx) >= val(fy)) {
        out[0] = {I, J, 1.0 - fx};
        out[1] = {I + 1, J, fx - fy};
        out[2] = {I + 1, J + 1, fy};
    } else {
        out[0] = {I, J, 1.0 - fy};
        out[1] = {I, J + 1, fy - fx};
        out[2] = {I + 1, J + 1, fx};
    }
}

/* ------------------------------------------------------------------------ */
/* Step 9 - gated Gaussian binomial (Sec. 6.3).                              */
/*   P>=1 = 1 - (1 - p)^N;  mu = (N-1) p;  sigma = sqrt((N-1) p (1-p));       */
/*   b ~ floor(gate * (1 + N(theta1; mu, sigma))).                           */
/* Readings: the gate succeeds with probability P>=1 (theta0 < P>=1: the     */
/* printed H(theta0 - P>=1) fires with the probability of zero successes);   */
/* N - 1 is clamped at 0 for fractional N < 1.  Sec. 6.3 builds the value as */
/* one guaranteed success (the gate) plus a Gaussian stand-in for            */
/* b(N-1, p), which is never negative: an open gate therefore counts at      */
/* least 1, and never more than ceil N, i.e. c = clamp(floor(1 + mu +        */
/* sigma z), 1, ceil N).  The relaxed count (for gradients) drops the floor. */
/* ------------------------------------------------------------------------ */
template <class T> struct CountLaw { T P1, mu, sigma; double nceil; };

template <class T>
CountLaw<T> count_law(const T& n, const T& p) {
    CountLaw<T> L;
    if (val(n) <= 0.0 || val(p) <= 0.0) L.P1 = T(0.0);
    else if (val(p) >= 1.0) L.P1 = T(1.0);
    else L.P1 = -expm1(n * log1p(-p));
    const T nm1 = val(n) > 1.0 ? n - 1.0 : T(0.0);
    L.mu = nm1 * p;
    const T var = L.mu * (1.0 - p);
    L.sigma = val(var) > 0.0 ? sqrt(var) : T(0.0);
    L.nceil = std::ceil(val(n));
    return L;
}

template <class T>
T gated_count(const CountLaw<T>& L, double th0, double th1, bool relaxed,
              int* gate, int* c_int, double* z, double* c_cont) {
    *gate = th0 < val(L.P1) ? 1 : 0;
    *z = 0.0; *c_cont = 0.0; *c_int = 0;
    if (!*gate) return T(0.0);
    *z = phi_inv(th1);
    const T cc = 1.0 + L.mu + L.sigma * (*z);
    *c_cont = val(cc);
    const double c = std::min(std::max(std::floor(val(cc)), 1.0), L.nceil);
    *c_int = c < 2147483647.0 ? (int)c : 2147483647;      /* trace value only */
    if (!relaxed) return T(c);
    if (val(cc) <= 1.0) return T(1.0);
    if (val(cc) >= L.nceil) return T(L.nceil);
    return cc;
}

/* Exact sampler (tests only): the count that the gated law stands in for,
 * the inverse of the Bin(N, p) cumulative distribution at theta for integer
 * N >= 0 - the smallest k with P(b <= k) > theta, the PMF summed from k = 0
 * in log space. */
int exact_binomial_count(int N, double p, double theta) {
    if (N <= 0 || p <= 0.0) return 0;
    if (p >= 1.0) return N;
    double cdf = 0.0;
    for (int k = 0; k < N; ++k) {
        cdf += std::exp(std::lgamma(N + 1.0) - std::lgamma(k + 1.0) - std::lgamma(N - k + 1.0) +
                        k * std::log(p) + (N - k) * std::log1p(-p));
        if (theta < cdf) return k;
    }
    return N;
}

/* Classical binomial approximation (Sec. 6.3, "Classical Binomial
 * Approximation"; the sampler the paper replaces): a Gaussian of the
 * binomial's own mean N p and variance N p (1 - p) sampled at theta0,
 * floored, where N p > 5; otherwise an explicit sum of Bernoulli trials.
 * Readings: a trial succeeds when theta_k < p (the printed H(theta_k - p)
 * fires with probability 1 - p, the sign slip of the gate); the loop runs
 * over at most 16 trials (Sec. 7.1: the compared implementation loops up to
 * N = 16), so N > 16 takes the Gaussian too; a fractional last trial
 * succeeds with probability p (N - floor N); the Gaussian count is clamped
 * to [0, ceil N].  The loop's uniforms come from the evaluation's second
 * word: theta_k of fmix32(h1 + k 0x9E3779B9), k = 1..ceil N.  *c_cont
 * receives the Gaussian's value, or the loop count plus 1/2 (never at an
 * integer: a loop count has no continuous value). */
constexpr int kClassicalLoopMax = 16;

template <class T>
T classical_count(const T& n, const T& p, uint32_t h0, uint32_t h1, int* c_int, double* z, double* c_cont) {
    const double nv = val(n), pv = val(p);
    *z = 0.0;
    if (nv <= 0.0 || pv <= 0.0) { *c_int = 0; *c_cont = 0.5; return T(0.0); }
    const double nceil = std::ceil(nv);
    if (nv * pv > 5.0 || nv > (double)kClassicalLoopMax) {
        const T mu = n * p;
        const T sig = sqrt(mu * (1.0 - p));
        *z = phi_inv(theta_of(h0));
        const T cc = mu + sig * (*z);
        *c_cont = val(cc);
        const double c = std::min(std::max(std::floor(val(cc)), 0.0), nceil);
        *c_int = c < 2147483647.0 ? (int)c : 2147483647;
        return T(c);
    }
    int c = 0;
    const int nt = (int)nceil;
    for (int k = 1; k <= nt; ++k) {
        const double pk = (k == nt && nceil != nv) ? pv * (nv - std::floor(nv)) : pv;
        if (theta_of(fmix32(h1 + (uint32_t)k * 0x9E3779B9u)) < pk) ++c;
    }
    *c_int = c;
    *c_cont = c + 0.5;
    return T((double)c);
}

/* Isotropic-grid mode (M = 0, Sec. 4 with manual anisotropic filtering): the
 * tetrahedron degenerates to the segment between the two LODs of the single
 * isotropic grid - vertex 0 (lower LOD, weight 1 - s) and vertex 3 (upper LOD,
 * weight s), the distributed binomial of Sec. 4.2 - and the two zero-weight
 * vertices 1, 2 are not evaluated: 2 x 3 x 4 = 24 evaluations per piece and
 * light instead of 48. */
static bool vertex_used(int M, int i) { return M > 0 || i == 0 || i == 3; }

/* ------------------------------------------------------------------------ */
/* Full pixel evaluation (Steps 1-10 in order).                              */
/* ------------------------------------------------------------------------ */
struct Seeds {             /* which tangents to seed (T = Dual only) */
    bool on;
    int light;             /* light whose direction is differentiated */
};

template <class T> void seed(T& x, int k, double dv);
template <> void seed<double>(double&, int, double) {}
template <> void seed<Dual>(Dual& x, int k, double dv) { x.d[k] = dv; }

template <class T>
T eval_pixel(const Scene& sc, int px, const Seeds& sd, bool relaxed, Trace* tr) {
    const OMaterial& M = sc.mat;
    const float* g = sc.gbuf + (size_t)px * 16;
    OPix info;
    std::memset(&info, 0, sizeof(info));
    auto finish = [&](int status, const T& out) {
        info.status = status;
        info.out = val(out);
        if (tr && tr->pix) *tr->pix = info;
        return out;
    };
    for (int k = 0; k < 15; ++k)
        if (!std::isfinite(g[k])) return finish(2, T(0.0));

    /* Step 1 - shading frame.  Background pixels carry n = 0. */
    const double u = g[0], v = g[1];
    const double dudx = g[2], dvdx = g[3], dudy = g[4], dvdy = g[5];
    double n[3] = {g[6], g[7], g[8]};
    double tg[3] = {g[9], g[10], g[11]};
    double wv[3] = {g[12], g[13], g[14]};
    if (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0) return finish(1, T(0.0));
    const double nl = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (double& c : n) c /= nl;
    const double tn = tg[0] * n[0] + tg[1] * n[1] + tg[2] * n[2];
    for (int k = 0; k < 3; ++k) tg[k] -= tn * n[k];
    const double tl = std::sqrt(tg[0] * tg[0] + tg[1] * tg[1] + tg[2] * tg[2]);
    const double vl = std::sqrt(wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2]);
    if (!(tl > 0.0) || !(vl > 0.0)) return finish(2, T(0.0));
    for (double& c : tg) c /= tl;
    for (double& c : wv) c /= vl;
    const double b[3] = {n[1] * tg[2] - n[2] * tg[1], n[2] * tg[0] - n[0] * tg[2], n[0] * tg[1] - n[1] * tg[0]};
    const double cos_v = wv[0] * n[0] + wv[1] * n[1] + wv[2] * n[2];
    if (!(cos_v > 0.0)) return finish(2, T(0.0));

    /* Material: scalar, or per-pixel (alpha, density) plane. */
    T ax, ay, rho;
    if (sc.mat_px) {
        const float* mp = sc.mat_px + (size_t)px * 2;
        ax = T((double)mp[0]); ay = T((double)mp[0]); rho = T((double)mp[1]);
    } else {
        ax = T((double)M.alpha_x); ay = T((double)M.alpha_y);
        T lr = T((double)M.ln_density);
        if (sd.on) { seed(ax, 0, 1.0); seed(ay, 1, 1.0); seed(lr, 2, 1.0); }
        rho = exp(lr);
    }

    /* Step 3 - footprint. */
    const Footprint fp = footprint(dudx, dudy, dvdx, dvdy);
    const T A = fp.P * rho;
    info.A = val(A); info.r = fp.r; info.phi = fp.phi; info.s0 = fp.s0; info.s1 = fp.s1;
    if (!(val(A) > 0.0)) return finish(2, T(0.0));

    /* Step 4 - sub-footprints. */
    const Split sp = split_footprint(fp.r, val(A), M.n_rings, M.n_lods, M.lod_factor, M.max_sub);
    info.K = sp.K; info.Kmaj = sp.Kmaj; info.k = sp.k;
    const T As = A / (double)sp.K;
    const double rho_r = std::log2(fp.r) - std::log2((double)sp.Kmaj);
    const double u0[2] = {std::cos(fp.phi), std::sin(fp.phi)};
    const double u1[2] = {-u0[1], u0[0]};

    /* Steps 5-7 per sub-footprint (independent of the light). */
    struct VertData {
        int level, ring, kor, upper; uint32_t gid; T w, n;
        SimplexVert<T> sv[3];
        T qx, qy;
    };
    struct SubData {
        Lod<T> lod; Cell cell; int tet; VertData vd[4];
    };
    SubData* subs = new SubData[sp.K];
    const int ncols = sp.Kmaj * sp.k;
    for (int sub = 0; sub < sp.K; ++sub) {
        const int ia = sub % ncols, ib = sub / ncols;
        const double oa = (ia + 0.5) / ncols - 0.5, ob = (ib + 0.5) / sp.k - 0.5;
        const double us = u + fp.s0 * oa * u0[0] + fp.s1 * ob * u1[0];
        const double vs = v + fp.s0 * oa * u0[1] + fp.s1 * ob * u1[1];
        SubData& S = subs[sub];
        S.lod = lod_bracket(As, M.lod_factor, M.n_lods);
        S.cell = ratio_cell(rho_r, fp.phi, M.n_rings);
        TetVert<T> tv[4];
        S.tet = tet_split(S.cell.lam, S.lod.s, tv);
        for (int i = 0; i < 4; ++i) {
            if (!vertex_used(M.n_rings, i)) continue;
            VertData& V = S.vd[i];
            V.upper = tv[i].upper;
            V.level = S.lod.level + tv[i].upper;
            V.ring = S.cell.v[tv[i].tv].ring;
            V.kor = S.cell.v[tv[i].tv].kor;
            V.gid = grid_id(V.level, V.ring, V.kor);
            V.w = tv[i].w;
            /* Trials: w_i times the cell's flake count f^level (Sec. 5.2,
             * "N_i proportional to its area"); pinned: w_i times A_s.  Linear
             * mix (Sec. 3, the scheme Sec. 4.2 replaces): every vertex counts
             * over its whole cell (f^level flakes; pinned: A_s) and its count
             * is weighted by w_i afterwards. */
            if (M.lod_blend == 1) V.n = S.lod.pinned ? As : T(std::pow((double)M.lod_factor, V.level));
            else V.n = S.lod.pinned ? V.w * As : V.w * std::pow((double)M.lod_factor, V.level);
            grid_coords(us, vs, V.level, V.ring, V.kor, rho, M.lod_factor, &V.qx, &V.qy);
            if (std::fabs(val(V.qx)) >= 0x1p30 || std::fabs(val(V.qy)) >= 0x1p30) {
                delete[] subs;
                return finish(3, T(0.0));
            }
            simplex_vertices(V.qx, V.qy, V.sv);
        }
    }

    /* Steps 8-10 per light. */
    T out = T(0.0);
    const T Dn = ndf_Dn(ax, ay);
    for (int l = 0; l < sc.nL; ++l) {
        const OLight& Lt = sc.lights[l];
        T wl[3], E;
        if (Lt.kind == 0) {
            const float* lp = sc.light_px + ((size_t)l * sc.W * sc.H + px) * 4;
            for (int k = 0; k < 3; ++k) wl[k] = T((double)lp[k]);
            E = T((double)lp[3]);
        } else {
            for (int k = 0; k < 3; ++k) wl[k] = T((double)Lt.dir[k]);
            E = T((double)Lt.intensity);
            if (sd.on && sd.light == l) for (int k = 0; k < 3; ++k) seed(wl[k], 3 + k, 1.0);
        }
        const T wll = sqrt(sq(wl[0]) + sq(wl[1]) + sq(wl[2]));
        if (!(val(wll) > 0.0)) continue;
        for (T& c : wl) c = c / wll;
        const T cos_l = wl[0] * n[0] + wl[1] * n[1] + wl[2] * n[2];
        if (!(val(cos_l) > 0.0)) continue;
        T hv[3];
        for (int k = 0; k < 3; ++k) hv[k] = wv[k] + wl[k];
        const T hl = sqrt(sq(hv[0]) + sq(hv[1]) + sq(hv[2]));
        for (T& c : hv) c = c / hl;
        const T ht = hv[0] * tg[0] + hv[1] * tg[1] + hv[2] * tg[2];
        const T hb = hv[0] * b[0] + hv[1] * b[1] + hv[2] * b[2];
        const T hn = hv[0] * n[0] + hv[1] * n[1] + hv[2] * n[2];

        /* Step 2 - Eq. 4: p = R D(h) / D(n), clamped to [0, 1]. */
        T p = (double)M.R * ndf_D(M.ndf, ax, ay, ht, hb, hn) / Dn;
        if (val(p) > 1.0) p = T(1.0);

        /* Step 8 (angular) - bilinear texels of the projected half-vector,
         * subdivided by the micro-roughness size gamma (Sec. 5.2, Eq. 14). */
        const T afx = ht / (double)M.gamma, afy = hb / (double)M.gamma;
        const double fax = std::floor(val(afx)), fay = std::floor(val(afy));
        const T fx = afx - fax, fy = afy - fay;
        const int32_t aX = (int32_t)fax, aY = (int32_t)fay;
        const int32_t axs[4] = {aX, aX + 1, aX, aX + 1};
        const int32_t ays[4] = {aY, aY, aY + 1, aY + 1};
        const T vw[4] = {(1.0 - fx) * (1.0 - fy), fx * (1.0 - fy), (1.0 - fx) * fy, fx * fy};

        /* Step 10 - C = sum over sub-footprints, tetrahedron vertices i,
         * simplex vertices j and angular texels k of u_ij v_k c_ijk (Eq. 14:
         * interpolate realisations; Eq. 10: distribute the trials). */
        T C = T(0.0);
        for (int sub = 0; sub < sp.K; ++sub) {
            const SubData& S = subs[sub];
            for (int i = 0; i < 4; ++i) {
                if (!vertex_used(M.n_rings, i)) continue;
                const VertData& V = S.vd[i];
                const CountLaw<T> law = count_law(V.n, p);
                for (int j = 0; j < 3; ++j) {
                    for (int k = 0; k < 4; ++k) {
                        uint32_t h0, h1;
                        if (M.rng_table == 1) eval_table(V.sv[j].i, V.sv[j].j, V.gid, axs[k], ays[k], M.seed, &h0, &h1);
                        else eval_hash(V.sv[j].i, V.sv[j].j, V.gid, axs[k], ays[k], M.seed, &h0, &h1);
                        int gate, ci; double z, ccont;
                        T c;
                        if (M.sampler == 1) {
                            gate = 1;
                            c = classical_count(V.n, p, h0, h1, &ci, &z, &ccont);
                        } else {
                            c = gated_count(law, theta_of(h0), theta_of(h1), relaxed, &gate, &ci, &z, &ccont);
                        }
                        if (M.lod_blend == 1) c = V.w * c;
                        C = C + V.sv[j].u * vw[k] * c;
                        if (tr && tr->recs) {
                            const int idx = tr->n++;
                            if (idx < tr->cap) {
                                ORec& R = tr->recs[idx];
                                R.light = l; R.sub = sub; R.vert = i; R.sv = j; R.av = k;
                                R.level = V.level; R.ring = V.ring; R.kor = V.kor;
                                R.tri = S.cell.tri; R.tet = S.tet; R.pinned = S.lod.pinned;
                                R.gid = V.gid; R.i = V.sv[j].i; R.j = V.sv[j].j;
                                R.ax = axs[k]; R.ay = ays[k]; R.h0 = h0; R.h1 = h1;
                                R.gate = gate; R.c = ci;
                                R.n = val(V.n); R.p = val(p); R.P1 = val(law.P1);
                                R.mu = val(law.mu); R.sigma = val(law.sigma); R.z = z; R.c_cont = ccont;
                                R.u = val(V.sv[j].u); R.v = val(vw[k]);
                                R.x = S.cell.x; R.t = S.cell.t; R.s = val(S.lod.s); R.As = val(As);
                                R.qx = val(V.qx); R.qy = val(V.qy); R.afx = val(afx); R.afy = val(afy);
                                R.w = val(V.w);
                            }
                        } else if (tr) {
                            tr->n++;
                        }
                    }
                }
            }
        }

        /* Eq. 3-4: D_P = D(n)/R * C / N(P).  Eq. 2 with Schlick F and
         * separable Smith G; L += rho_P * E * cos_l. */
        const T DP = Dn / (double)M.R * C / A;
        const T vh = wv[0] * hv[0] + wv[1] * hv[1] + wv[2] * hv[2];
        const T om = 1.0 - vh;
        const T F = (double)M.F0 + (1.0 - (double)M.F0) * sq(sq(om)) * om;
        const T lam_v = smith_lambda(M.ndf, ax, ay, T(wv[0] * tg[0] + wv[1] * tg[1] + wv[2] * tg[2]),
                                     T(wv[0] * b[0] + wv[1] * b[1] + wv[2] * b[2]), T(cos_v));
        const T wlt = wl[0] * tg[0] + wl[1] * tg[1] + wl[2] * tg[2];
        const T wlb = wl[0] * b[0] + wl[1] * b[1] + wl[2] * b[2];
        const T lam_l = smith_lambda(M.ndf, ax, ay, wlt, wlb, cos_l);
        const T G = 1.0 / ((1.0 + lam_v) * (1.0 + lam_l));
        out = out + F * G * DP / (4.0 * cos_v * cos_l) * E * cos_l;
    }
    delete[] subs;
    return finish(0, out);
}

int check_material(const OMaterial* m, int nL) {
    if (!m) return -1;
    if (m->ndf != 0 && m->ndf != 1) return -1;
    if (m->n_lods < 2 || m->n_lods > 16) return -1;
    if (m->n_rings < 0 || m->n_rings > 6) return -1;
    if (m->lod_factor != 2 && m->lod_factor != 4) return -1;
    if (m->max_sub < 1 || m->max_sub > 64) return -1;
    if (!(m->R > 0.0f && m->R <= 1.0f) || !(m->gamma >= 1e-3f)) return -1;
    if (nL < 0 || nL > 8) return -1;
    if ((m->lod_blend != 0 && m->lod_blend != 1) || (m->sampler != 0 && m->sampler != 1)) return -1;
    if (m->rng_table != 0 && m->rng_table != 1) return -1;
    return 0;
}

Scene make_scene(const float* gbuf, const float* light_px, const float* mat_px, int W, int H,
                 const OMaterial* mat, const OLight* lights, int nL) {
    Scene s;
    s.gbuf = gbuf; s.light_px = light_px; s.mat_px = mat_px; s.W = W; s.H = H; s.nL = nL;
    s.mat = *mat; s.lights = lights;
    return s;
}

void set_threads(int n_threads) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
}

}  // namespace

/* ======================================================================== */
/* C entry points (ctypes).                                                  */
/* ======================================================================== */
extern "C" {

int oracle_struct_sizes(int32_t* out4) {
    out4[0] = (int32_t)sizeof(OMaterial); out4[1] = (int32_t)sizeof(OLight);
    out4[2] = (int32_t)sizeof(OPix); out4[3] = (int32_t)sizeof(ORec);
    return 0;
}

/* Image (or pixel list) evaluation.  out[i] = radiance of pixel px_list[i]
 * (or of pixel i when px_list is null, n_px = W*H).  relaxed != 0 gives the
 * relaxed-count image used by finite differences. */
int oracle_eval(const float* gbuf, const float* light_px, const float* mat_px, int W, int H,
                const OMaterial* mat, const OLight* lights, int nL,
                const int32_t* px_list, int n_px, int relaxed, double* out, int n_threads) {
    if (!gbuf || !out || W <= 0 || H <= 0 || check_material(mat, nL)) return -1;
    const Scene sc = make_scene(gbuf, light_px, mat_px, W, H, mat, lights, nL);
    const int count = px_list ? n_px : W * H;
    set_threads(n_threads);
    const Seeds sd = {false, -1};
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < count; ++i) {
        const int px = px_list ? px_list[i] : i;
        out[i] = eval_pixel<double>(sc, px, sd, relaxed != 0, nullptr);
    }
    return 0;
}

/* Parity trace of one pixel: summary plus every binomial evaluation in the
 * canonical order (light, sub-footprint, tetrahedron vertex, simplex vertex,
 * angular texel).  *n_rec receives the total record count (may exceed cap). */
int oracle_trace(const float* gbuf, const float* light_px, const float* mat_px, int W, int H,
                 const OMaterial* mat, const OLight* lights, int nL, int px,
                 OPix* pix, ORec* recs, int cap, int* n_rec) {
    if (!gbuf || !pix || check_material(mat, nL) || px < 0 || px >= W * H) return -1;
    const Scene sc = make_scene(gbuf, light_px, mat_px, W, H, mat, lights, nL);
    Trace tr = {pix, recs, cap, 0};
    const Seeds sd = {false, -1};
    eval_pixel<double>(sc, px, sd, false, &tr);
    if (n_rec) *n_rec = tr.n;
    return 0;
}

/* FP64 gradient of sum_px grad_out[px] * relaxed_out[px] with respect to
 * (alpha_x, alpha_y, ln density, direction of light grad_light).  Requires
 * the scalar material (no per-pixel plane).  per_px (n_px x 6) and
 * relaxed (n_px) are optional. */
int oracle_grad(const float* gbuf, const float* light_px, int W, int H,
                const OMaterial* mat, const OLight* lights, int nL, int grad_light,
                const int32_t* px_list, int n_px, const double* grad_out,
                double* grad6, double* per_px, double* relaxed, int n_threads) {
    if (!gbuf || !grad6 || !grad_out || check_material(mat, nL)) return -1;
    const Scene sc = make_scene(gbuf, light_px, nullptr, W, H, mat, lights, nL);
    const int count = px_list ? n_px : W * H;
    set_threads(n_threads);
    const Seeds sd = {true, grad_light};
    for (int k = 0; k < NG; ++k) grad6[k] = 0.0;
    double acc[NG] = {0, 0, 0, 0, 0, 0};
#pragma omp parallel
    {
        double loc[NG] = {0, 0, 0, 0, 0, 0};
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < count; ++i) {
            const int px = px_list ? px_list[i] : i;
            const Dual o = eval_pixel<Dual>(sc, px, sd, true, nullptr);
            for (int k = 0; k < NG; ++k) loc[k] += grad_out[i] * o.d[k];
            if (per_px) for (int k = 0; k < NG; ++k) per_px[(size_t)i * NG + k] = o.d[k];
            if (relaxed) relaxed[i] = o.v;
        }
#pragma omp critical
        for (int k = 0; k < NG; ++k) acc[k] += loc[k];
    }
    for (int k = 0; k < NG; ++k) grad6[k] = acc[k];
    return 0;
}

/* ---- pieces exported for unit tests ------------------------------------ */
double oracle_phi_inv(double P) { return phi_inv(P); }

void oracle_pcg4d(uint32_t* v) { pcg4d(v); }
void oracle_pcg3d(uint32_t* v) { pcg3d(v); }
uint32_t oracle_fmix32(uint32_t h) { return fmix32(h); }
uint32_t oracle_grid_id(int level, int ring, int kor) { return grid_id(level, ring, kor); }
void oracle_eval_hash(int32_t i, int32_t j, uint32_t gid, int32_t ax, int32_t ay, uint32_t seed, uint32_t* h2) {
    eval_hash(i, j, gid, ax, ay, seed, &h2[0], &h2[1]);
}
double oracle_theta(uint32_t h) { return theta_of(h); }
void oracle_table_words(uint32_t k, uint32_t* h2) { table_words(k, &h2[0], &h2[1]); }
void oracle_eval_table(int32_t i, int32_t j, uint32_t gid, int32_t ax, int32_t ay, uint32_t seed, uint32_t* h2) {
    eval_table(i, j, gid, ax, ay, seed, &h2[0], &h2[1]);
}

double oracle_ndf(int ndf, double ax, double ay, double ht, double hb, double hn) {
    return ndf_D<double>(ndf, ax, ay, ht, hb, hn);
}
double oracle_smith_lambda(int ndf, double ax, double ay, double wt, double wb, double wn) {
    return smith_lambda<double>(ndf, ax, ay, wt, wb, wn);
}

/* out5 = (sigma0, sigma1, phi, P, r) */
void oracle_footprint(double a, double b, double c, double d, double* out5) {
    const Footprint f = footprint(a, b, c, d);
    out5[0] = f.s0; out5[1] = f.s1; out5[2] = f.phi; out5[3] = f.P; out5[4] = f.r;
}

/* out3 = (Kmaj, k, K) */
void oracle_split(double r, double A, int M, int L, int f, int Kmax, int32_t* out3) {
    const Split s = split_footprint(r, A, M, L, f, Kmax);
    out3[0] = s.Kmaj; out3[1] = s.k; out3[2] = s.K;
}

/* iout = (level, pinned); dout = (s) */
void oracle_lod(double As, int f, int L, int32_t* iout, double* dout) {
    const Lod<double> l = lod_bracket<double>(As, f, L);
    iout[0] = l.level; iout[1] = l.pinned ? 1 : 0; dout[0] = l.s;
}

/* iout = (m, tri, ring0, kor0, ring1, kor1, ring2, kor2); dout = (x, t, lam0, lam1, lam2) */
void oracle_cell(double rho_r, double phi, int M, int32_t* iout, double* dout) {
    const Cell c = ratio_cell(rho_r, phi, M);
    iout[0] = c.m; iout[1] = c.tri;
    for (int k = 0; k < 3; ++k) { iout[2 + 2 * k] = c.v[k].ring; iout[3 + 2 * k] = c.v[k].kor; }
    dout[0] = c.x; dout[1] = c.t; dout[2] = c.lam[0]; dout[3] = c.lam[1]; dout[4] = c.lam[2];
}

/* iout = (tet, upper0, tv0, upper1, tv1, ...); wout = 4 weights */
void oracle_tet(const double* lam3, double s, int32_t* iout, double* wout) {
    TetVert<double> tv[4];
    iout[0] = tet_split<double>(lam3, s, tv);
    for (int k = 0; k < 4; ++k) { iout[1 + 2 * k] = tv[k].upper; iout[2 + 2 * k] = tv[k].tv; wout[k] = tv[k].w; }
}

void oracle_grid_coords(double u, double v, int level, int ring, int kor, double rho, int f, double* q2) {
    grid_coords<double>(u, v, level, ring, kor, rho, f, &q2[0], &q2[1]);
}

/* iout = (i0, j0, i1, j1, i2, j2); wout = 3 weights */
void oracle_simplex(double qx, double qy, int32_t* iout, double* wout) {
    SimplexVert<double> s[3];
    simplex_vertices<double>(qx, qy, s);
    for (int k = 0; k < 3; ++k) { iout[2 * k] = s[k].i; iout[2 * k + 1] = s[k].j; wout[k] = s[k].u; }
}

/* Classical count of one evaluation (words h0, h1).  dout = (z, c_cont); returns c. */
int oracle_classical_count(double n, double p, uint32_t h0, uint32_t h1, double* dout) {
    int c; double z, cc;
    classical_count<double>(n, p, h0, h1, &c, &z, &cc);
    dout[0] = z; dout[1] = cc;
    return c;
}

/* Exact binomial count (inverse CDF) of one evaluation. */
int oracle_exact_count(int N, double p, double theta) { return exact_binomial_count(N, p, theta); }

/* Gated count of one evaluation.  dout = (P1, mu, sigma, z, c_cont, relaxed); returns c. */
int oracle_gated_count(double n, double p, double th0, double th1, double* dout) {
    const CountLaw<double> L = count_law<double>(n, p);
    int gate, c; double z, cc;
    const double rel = gated_count<double>(L, th0, th1, true, &gate, &c, &z, &cc);
    dout[0] = L.P1; dout[1] = L.mu; dout[2] = L.sigma; dout[3] = z; dout[4] = cc; dout[5] = rel;
    return c;
}

}  // extern "C"
