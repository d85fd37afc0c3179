// Plain forward kernel (one frame) and the parity-trace kernel.
//
// Forward kernel mapping: one warp shades 32 pixels of its CTA's tile (lane =
// pixel, 8 groups of 4 consecutive pixels, see tile_pixel) for the
// per-pixel, per-light and per-sub-footprint setup, then walks
// the evaluations in a warp-uniform loop (sub-footprint, light, 4 grids x 3
// simplex vertices x 4 angular texels).  Each lane tests its gate with one
// hash word; the rare open gates (their count needs the second word, a normal
// quantile and the floor) are appended to a per-warp queue in shared memory
// and evaluated 32 at a time at full warp width, so that the divergent,
// expensive part of the binomial law costs one lane-slot per open gate
// rather than a warp-slot.  Results are returned to their owner lanes in
// enqueue order, so the image is deterministic.
#include <mutex>
#include "glint_kernels.cuh"

namespace glint {

constexpr int kQ = 64;                    // queue capacity per warp (ring)

// --------------------------------------------------------------------------
// random-number table (Sec. 6.3, last paragraph; rng_table = 1): 2^16 pairs
// of words, R[k] = (fmix32(2k G + C), fmix32((2k + 1) G + C)), G = 0x9E3779B9,
// C = 0x632BE5AB, filled once per device on first use.  An evaluation with
// spatial word s and angular word a reads R[(s + a) >> 16] in place of the
// two per-evaluation mixing steps.
// --------------------------------------------------------------------------
constexpr int kRngTableBits = 16;
static __device__ uint2 g_rng_table[1 << kRngTableBits];

__device__ __forceinline__ uint2 rng_table_pair(uint32_t key) {
    return __ldg(&g_rng_table[key >> (32 - kRngTableBits)]);
}

__global__ void rng_table_kernel() {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < (1u << kRngTableBits))
        g_rng_table[k] = make_uint2(fmix32(2u * k * 0x9E3779B9u + 0x632BE5ABu),
                                    fmix32((2u * k + 1u) * 0x9E3779B9u + 0x632BE5ABu));
}

// Fill the table once per device: one kernel on `s`, then a wait for it, so
// that work on any stream may read the table afterwards.
cudaError_t ensure_rng_table(cudaStream_t s) {
    static std::mutex mtx;
    static bool done[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mtx);
    if (done[dev]) return cudaSuccess;
    rng_table_kernel<<<(1 << kRngTableBits) / 256, 256, 0, s>>>();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    done[dev] = true;
    return cudaSuccess;
}

struct WarpQueue {
    uint32_t word[kQ];                    // pre-image of the second hash word
    float mu[kQ], mu_lo[kQ], sig[kQ], nceil[kQ], w[kQ];
    int32_t owner[kQ];
    float res[32];
    uint32_t mask[32];
};
// (its first 16 x 32 words also hold the lanes' shading frames, SharedFrame)
static_assert(sizeof(WarpQueue) >= 16 * 32 * sizeof(float), "warp queue too small for the frame words");

// Copy the double-float tables (only the rotation entries up to ring M)
// from the parameter block into shared memory (trace kernel).  The image
// kernels read them in the parameter block itself, through the constant
// cache: the shared copy's 9.5 KB per CTA are worth more as L1 for the
// per-thread stack (two CTAs then fit the 164 KB shared configuration, which
// leaves ~92 KB of L1 per SM instead of ~60 KB).
__device__ __forceinline__ void load_tables(const KParams& P, Tables& T) {
    const int nwords = tables_words(P.M);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&P.tables);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&T);
    for (int k = threadIdx.x; k < nwords; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// Evaluate the n <= 32 queue entries starting at `head`: lane k takes entry
// head + k.  Each owner lane then adds its entries' values in queue order to
// its running sum, which goes in and comes back by value (a reference would
// send it through the stack at every call).
// kFinal: the queue holds the second hash word itself (table mode), else
// its pre-image.
template <bool kFinal>
__device__ __noinline__ float flush_queue(WarpQueue& q, int head, int n, float acc) {
    const int lane = threadIdx.x & 31;
    const int e = (head + lane) & (kQ - 1);
    float val = 0.0f;
    int owner = 32 + lane;                       // unique dummy for empty slots
    if (lane < n) {
        float cc;
        const uint32_t h1 = kFinal ? q.word[e] : fmix32(q.word[e]);
        val = q.w[e] * open_count(h1, q.mu[e], q.mu_lo[e], q.sig[e], q.nceil[e], &cc);
        owner = q.owner[e];
    }
    q.res[lane] = val;
    q.mask[lane] = 0u;
    __syncwarp();
    const unsigned grp = __match_any_sync(0xffffffffu, owner);
    if (lane < n && lane == __ffs(grp) - 1) q.mask[owner] = grp;
    __syncwarp();
    unsigned mine = q.mask[lane];
    while (mine) {
        const int k = __ffs(mine) - 1;
        acc += q.res[k];
        mine &= mine - 1;
    }
    __syncwarp();
    return acc;
}

struct LightEval {          // what the evaluation loop needs of one light
    bool on;
    float p, p_lo, lq, shade;
    float v[4];
    uint32_t A0[4], A1[4];
};

// Shade the pixel of this lane (px valid or not); all 32 lanes call together.
// ss0 / suw: the CTA's shared arrays of 12 x blockDim spatial words / weights.
// kMode (kernel_variant): kRing the anisotropic grids; kIsoGrid the
// isotropic-grid mode (M = 0), tetrahedron vertices 0 and 3 only;
// kClassicalSampler the classical sampler (ablation, sampler = 1), evaluated
// by each lane for its own pixel (every evaluation draws a count: no gate,
// no queue), M = 0 handled at run time; kRngTable the uniforms fetched from
// the random-number table instead of the per-evaluation mixing.
template <int kMode>
__device__ float shade_warp(const KParams& P, const Tables& T, const FrameDesc& F, WarpQueue& q, int px,
                            bool valid, uint32_t* ss0, float* suw) {
    constexpr bool kIso = kMode == kIsoGrid, kClassical = kMode == kClassicalSampler, kTable = kMode == kRngTable;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    PixelSetup S;
    S.status = 1;
    S.K = 0;
    // the shading frame lives in this lane's slots of the warp's queue and
    // spatial words until the lights are set up
    const SharedFrame R{reinterpret_cast<float*>(&q) + lane, reinterpret_cast<float*>(ss0) + threadIdx.x,
                        (int)blockDim.x};
    if (valid) setup_pixel<false>(P, T, F, px, S, R);
    LightState ls[kMaxLights];
    bool any_on = false;
    // the largest trial count of the tetrahedron: P>=1 grows with N, so a
    // light whose gates cannot open at this count (P>=1 <= 2^-26, half of the
    // gate's resolution) opens none at any vertex and adds nothing
    const float n_max = fmaxf(fmaxf(S.ntr[0], S.ntr[1]), fmaxf(S.ntr[2], S.ntr[3]));
    for (int l = 0; l < F.nL; ++l) {
        ls[l].on = false;
        if (S.status == 0) setup_light<false, SharedFrame, false>(P, T, F, S, R, px, l, ls[l]);
        if (ls[l].on && ls[l].p < 1.0f && !kClassical && -expm1f(n_max * ls[l].lq) <= 1.4901161193847656e-8f)
            ls[l].on = false;
        any_on |= ls[l].on;
    }
    __syncwarp();   // the frame's slots go back to the queue and the spatial words
    // a pixel that no light reaches, or whose gates cannot open, shades to 0:
    // its sub-footprints are not set up
    const int K = S.status == 0 && any_on ? S.K : 0;
    const int Kw = __reduce_max_sync(0xffffffffu, K);
    float acc = 0.0f;
    int head = 0, count = 0;                     // warp-uniform queue state
    bool in_range = true;
    // this lane's 12 spatial words and weights, structure-of-arrays in shared memory
    uint32_t* s0s = ss0 + threadIdx.x;
    float* uws = suw + threadIdx.x;
    const int st = blockDim.x;
    for (int sub = 0; sub < Kw; ++sub) {
        SubState U;
        bool act = sub < K && in_range;
        if (act) {
            // (the classical variant runs both grid modes: with M = 0 only
            // vertices 0 and 3 exist, and only the M = 0 rotation entry is loaded)
            in_range = (kClassical && P.M == 0) ? setup_sub<false, true>(P, T, S, sub, U, s0s, uws, st)
                                                : setup_sub<false, kIso>(P, T, S, sub, U, s0s, uws, st);
            act = in_range;
        }
#pragma unroll 1
        for (int l = 0; l < F.nL; ++l) {
            LightEval L;
            L.on = act && ls[l].on;
            L.p = ls[l].p; L.p_lo = ls[l].p_lo; L.lq = ls[l].lq; L.shade = ls[l].shade;
#pragma unroll
            for (int k = 0; k < 4; ++k) L.v[k] = ls[l].v[k];
            if (!__any_sync(0xffffffffu, L.on)) continue;
            // the angular words are formed here from the texel rather than
            // stored per light (less stack)
            angular_words(P, ls[l].ix0, ls[l].iy0, L.A0, L.A1);
#pragma unroll 1
            for (int ii = 0; ii < (kIso ? 2 : 4); ++ii) {
                const int i = kIso ? 3 * ii : ii;
                const float shade_i = P.lod_blend ? L.shade * S.wmix[i] : L.shade;   // linear-mix ablation
                if (kClassical) {
                    if (!vertex_used(P.M, i) || !L.on) continue;
                    const ClassicalLaw cl = classical_law(S.ntr[i], S.ntr_lo[i], L.p, L.p_lo);
#pragma unroll 1
                    for (int j = 0; j < 3; ++j) {
                        const uint32_t s0 = s0s[(3 * i + j) * st], s1 = U.S1[3 * i + j];
                        const float uw = uws[(3 * i + j) * st] * shade_i;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            float cc;
                            acc += uw * L.v[k] * classical_count(cl, fmix32(s0 + L.A0[k]), fmix32(s1 + L.A1[k]), &cc);
                        }
                    }
                    continue;
                }
                CountLaw law = count_law(S.ntr[i], S.ntr_lo[i], L.p, L.p_lo, L.lq);
                if (!L.on) law.Tg = 0u;
                // no gate of this grid can open in any lane (P>=1 below 2^-25,
                // e.g. a half-vector far from the NDF's peak): its 12
                // evaluations add nothing
                if (!__any_sync(0xffffffffu, law.Tg > 1u)) continue;
                // (not unrolled: three copies of the queue-push code cost more
                // in instruction-cache misses than the loop does)
#pragma unroll 1
                for (int j = 0; j < 3; ++j) {
                    const uint32_t s0 = s0s[(3 * i + j) * st], s1 = U.S1[3 * i + j];
                    const float uw = uws[(3 * i + j) * st] * shade_i;
                    // one warp vote for the 4 angular texels: most groups have no open gate
                    bool gk[4];
                    uint32_t w1[4];                   // table mode: the second words, fetched with the first
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        uint32_t h0;
                        if (kTable) {
                            const uint2 t = rng_table_pair(s0 + L.A0[k]);
                            h0 = t.x; w1[k] = t.y;
                        } else {
                            h0 = fmix32(s0 + L.A0[k]);
                            w1[k] = s1 + L.A1[k];
                        }
                        gk[k] = gate_open(h0, law.Tg);
                    }
                    if (!__any_sync(0xffffffffu, gk[0] | gk[1] | gk[2] | gk[3])) continue;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool g = gk[k];
                        const unsigned m = __ballot_sync(0xffffffffu, g);
                        if (m) {
                            if (g) {
                                const int pos = (head + count + __popc(m & lt_mask)) & (kQ - 1);
                                q.word[pos] = w1[k];
                                q.mu[pos] = law.mu; q.mu_lo[pos] = law.mu_lo;
                                q.sig[pos] = law.sig; q.nceil[pos] = law.nceil;
                                q.w[pos] = uw * L.v[k];
                                q.owner[pos] = lane;
                            }
                            count += __popc(m);
                            if (count >= 32) {
                                __syncwarp();
                                acc = flush_queue<kTable>(q, head, 32, acc);
                                head = (head + 32) & (kQ - 1);
                                count -= 32;
                            }
                        }
                    }
                }
            }
        }
    }
    if (count > 0) {
        __syncwarp();
        acc = flush_queue<kTable>(q, head, count, acc);
    }
    if (S.status != 0 || !in_range) return 0.0f;
    return acc / S.A.hi;
}

// Pixel of this thread in a tile of blockDim.x pixels: lanes take groups of 4
// consecutive pixels spread over the whole tile (warp w, lane l -> group
// (l / 4) * warps + w).  Neighbouring pixels cost about the same (same lights
// on, same flake density), so spreading each warp over the tile evens out
// the warps' work, and the warps wait less at the tile barrier.
__device__ __forceinline__ int tile_pixel() {
    const int nw = (int)blockDim.x >> 5;
    const int ln = (int)threadIdx.x & 31, w = (int)threadIdx.x >> 5;
    return (ln >> 2) * (nw * 4) + w * 4 + (ln & 3);
}

// 2-D tiles: a block of kTileW x (threads / kTileW) pixels per CTA instead of
// a run of consecutive pixels of one row.  A compact block holds pixels of
// similar cost, so the CTA's warps finish closer together; on the 4K sphere
// frame this is 14% faster than row tiles.  The plain kernel is instantiated
// for each tiling (k2D), the batched one takes it per frame at run time.  A frame with few tiles keeps row
// tiles: with few waves of CTAs, compact blocks would gather its expensive
// region (a highlight) into few CTAs, which then set the launch's length.
#ifndef GLINT_TILE_W
#define GLINT_TILE_W 16
#endif
constexpr int kTileW = GLINT_TILE_W;
constexpr int kMin2DTiles = 2048;          // row tiles of a frame needed before 2-D tiles are used

int frame_tiles(FrameDesc& F, int threads) {
    const long long rows1d = ((long long)F.npx + threads - 1) / threads;
    const int th = threads / kTileW;
    F.tile_w = (rows1d >= kMin2DTiles && threads % kTileW == 0 && F.W >= 4 * kTileW && F.H >= 4 * th) ? kTileW : 0;
    if (!F.tile_w) return (int)rows1d;
    return ((F.W + kTileW - 1) / kTileW) * ((F.H + th - 1) / th);
}

// Pixel of this thread (tile-local index i = tile_pixel()) in tile t of frame
// F, or -1 where the tile overhangs the frame.  tile_w is 0 or kTileW, so the
// 2-D offsets divide by a constant.
__device__ __forceinline__ int tile_px(const FrameDesc& F, int t, int i) {
    if (F.tile_w == 0) {
        const int px = t * (int)blockDim.x + i;
        return px < F.npx ? px : -1;
    }
    const int th = (int)blockDim.x / kTileW;
    const int tiles_x = (F.W + kTileW - 1) / kTileW;
    const int ty = t / tiles_x;
    const int x = (t - ty * tiles_x) * kTileW + i % kTileW, y = ty * th + i / kTileW;
    return (x < F.W && y < F.H) ? y * F.W + x : -1;
}

__device__ __forceinline__ int tile_px_1d(const FrameDesc& F, int t, int i) {
    const int px = t * (int)blockDim.x + i;
    return px < F.npx ? px : -1;
}
__device__ __forceinline__ int tile_px_2d(const FrameDesc& F, int t, int i) {
    const int th = (int)blockDim.x / kTileW;
    const int tiles_x = (F.W + kTileW - 1) / kTileW;
    const int ty = t / tiles_x;
    const int x = (t - ty * tiles_x) * kTileW + i % kTileW, y = ty * th + i / kTileW;
    return (x < F.W && y < F.H) ? y * F.W + x : -1;
}
__device__ __forceinline__ int tile_count_1d(const FrameDesc& F) { return (F.npx + (int)blockDim.x - 1) / (int)blockDim.x; }
__device__ __forceinline__ int tile_count_2d(const FrameDesc& F) {
    const int th = (int)blockDim.x / kTileW;
    return ((F.W + kTileW - 1) / kTileW) * ((F.H + th - 1) / th);
}

template <int kMode, bool k2D>
__global__ void __launch_bounds__(1024) fwd_kernel(const __grid_constant__ KParams P, const FrameDesc F) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Tables& T = P.tables;
    WarpQueue* Qs = reinterpret_cast<WarpQueue*>(smem);
    uint32_t* ss0 = reinterpret_cast<uint32_t*>(Qs + blockDim.x / 32);
    float* suw = reinterpret_cast<float*>(ss0 + 12 * blockDim.x);
    WarpQueue& q = Qs[threadIdx.x >> 5];
    // Block-uniform tiles of blockDim.x pixels.  The barrier at the top of a
    // tile keeps the block's warps together in the (long, mostly
    // straight-line) setup code so they share instruction-cache lines.
    // (the tile count and offsets are recomputed from the parameters each
    // tile: nothing extra stays live across the shading, which fills the
    // 64 registers)
    for (int t = blockIdx.x; t < (k2D ? tile_count_2d(F) : tile_count_1d(F)); t += gridDim.x) {
        __syncthreads();
        const int px = k2D ? tile_px_2d(F, t, tile_pixel()) : tile_px_1d(F, t, tile_pixel());
        const float o = shade_warp<kMode>(P, T, F, q, px < 0 ? 0 : px, px >= 0, ss0, suw);
        if (px >= 0) __stcs(F.out + px, o);
    }
}

// Kernel over the tiles of many frames; tile t belongs to frame f with
// tile_base[f] <= t < tile_base[f+1].  Persistent: CTAs take tiles from a
// global counter (reset to 0 before the launch).  Otherwise one CTA per tile
// (CTA b shades tile b), scheduled by the hardware.
template <int kMode>
__global__ void __launch_bounds__(1024) batch_kernel(const __grid_constant__ KParams P,
                                                     const __grid_constant__ BatchDesc B) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Tables& T = P.tables;
    WarpQueue* Qs = reinterpret_cast<WarpQueue*>(smem);
    uint32_t* ss0 = reinterpret_cast<uint32_t*>(Qs + blockDim.x / 32);
    float* suw = reinterpret_cast<float*>(ss0 + 12 * blockDim.x);
    __shared__ int tile_s;
    WarpQueue& q = Qs[threadIdx.x >> 5];
    for (int it = 0;; ++it) {
        __syncthreads();
        if (threadIdx.x == 0)
            tile_s = B.persistent ? (int)atomicAdd(B.counter, 1u) : (it == 0 ? (int)blockIdx.x : 0x7fffffff);
        __syncthreads();
        const int t = tile_s;
        if (t >= B.tile_base[B.n]) break;
        int lo = 0, hi = B.n - 1;                 // last frame with tile_base <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.tile_base[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const FrameDesc& F = B.frames[lo];
        const int px = tile_px(F, t - B.tile_base[lo], tile_pixel());
        const float o = shade_warp<kMode>(P, T, F, q, px < 0 ? 0 : px, px >= 0, ss0, suw);
        if (px >= 0) __stcs(F.out + px, o);
    }
}

size_t fwd_smem_bytes(int threads) {
    return (size_t)(threads / 32) * sizeof(WarpQueue) + (size_t)threads * 24 * sizeof(uint32_t);
}

// --------------------------------------------------------------------------
// parity trace: one thread per listed pixel, every evaluation recorded
// --------------------------------------------------------------------------
__device__ void trace_pixel(const KParams& P, const Tables& T, const FrameDesc& F, int px, GlintTracePix* pr,
                            GlintTraceRec* recs, int cap) {
    PixelSetup S;
    LocalFrame R;
    setup_pixel<true>(P, T, F, px, S, R);
    pr->status = S.status; pr->K = S.status == 0 ? S.K : 0; pr->n_rec = 0; pr->n_can_open = 0;
    pr->A = S.status == 0 ? S.A.hi : 0.0f; pr->r = S.status == 0 ? S.ratio.hi : 0.0f;
    pr->phi = S.status == 0 ? S.phi.hi : 0.0f; pr->out = 0.0f;
    if (S.status != 0) return;
    LightState ls[kMaxLights];
    for (int l = 0; l < F.nL; ++l) setup_light<true>(P, T, F, S, R, px, l, ls[l]);
    float C[kMaxLights];
    for (int l = 0; l < F.nL; ++l) C[l] = 0.0f;
    int nrec = 0, ncan = 0;
    for (int sub = 0; sub < S.K; ++sub) {
        SubState U;
        const bool ok = P.M > 0 ? setup_sub<true, false>(P, T, S, sub, U, U.S0, U.uw, 1)
                                : setup_sub<true, true>(P, T, S, sub, U, U.S0, U.uw, 1);
        if (!ok) { pr->status = 3; pr->n_rec = nrec; pr->n_can_open = ncan; return; }
        for (int l = 0; l < F.nL; ++l) {
            const LightState& L = ls[l];
            if (!L.on) continue;
            for (int i = 0; i < 4; ++i) {
                if (!vertex_used(P.M, i)) continue;
                const CountLaw law = count_law(S.ntr[i], S.ntr_lo[i], L.p, L.p_lo, L.lq);
                const ClassicalLaw cl = classical_law(S.ntr[i], S.ntr_lo[i], L.p, L.p_lo);
                for (int j = 0; j < 3; ++j) {
                    for (int k = 0; k < 4; ++k) {
                        uint32_t h0, h1;
                        if (P.rng_table) {
                            const uint2 t = rng_table_pair(U.S0[3 * i + j] + L.A0[k]);
                            h0 = t.x; h1 = t.y;
                        } else {
                            h0 = fmix32(U.S0[3 * i + j] + L.A0[k]);
                            h1 = fmix32(U.S1[3 * i + j] + L.A1[k]);
                        }
                        bool g;
                        float c = 0.0f, cc = 0.0f;
                        if (P.sampler) {
                            g = true;                             // every evaluation draws a count
                            c = classical_count(cl, h0, h1, &cc);
                        } else {
                            g = gate_open(h0, law.Tg);
                            if (g) c = open_count(h1, law.mu, law.mu_lo, law.sig, law.nceil, &cc);
                        }
                        if (g) C[l] += U.uw[3 * i + j] * L.v[k] * (S.wmix[i] * c);
                        const int idx = (((l * S.K + sub) * 4 + i) * 3 + j) * 4 + k;
                        ++nrec;
                        ncan += (P.sampler || law.Tg > 1u) ? 1 : 0;
                        if (idx < cap) {
                            GlintTraceRec& R = recs[idx];
                            R.light = l; R.sub = sub; R.vert = i; R.sv = j; R.av = k; R.grid_id = U.gid[i];
                            R.i = U.li[3 * i + j]; R.j = U.lj[3 * i + j]; R.ax = L.ax[k]; R.ay = L.ay[k];
                            R.h0 = h0; R.h1 = h1; R.gate = g ? 1 : 0;
                            R.c = c < 2147483647.0f ? (int)c : 2147483647;
                            R.n = S.ntr[i]; R.P1 = P.sampler ? 1.0f : law.P1;
                            R.mu = P.sampler ? cl.mu : law.mu; R.sigma = P.sampler ? cl.sig : law.sig; R.c_cont = cc;
                            R.u = U.uw[3 * i + j]; R.v = L.v[k]; R.p = L.p;
                        }
                    }
                }
            }
        }
    }
    float out = 0.0f;
    for (int l = 0; l < F.nL; ++l)
        if (ls[l].on) out += ls[l].shade * C[l];
    pr->out = out / S.A.hi;
    pr->n_rec = nrec;
    pr->n_can_open = ncan;
}

__global__ void __launch_bounds__(128) trace_kernel(const __grid_constant__ KParams P, const FrameDesc F,
                                                    const int32_t* px_list, int32_t n_px, GlintTracePix* pix,
                                                    GlintTraceRec* recs, int32_t cap) {
    __shared__ Tables T;
    load_tables(P, T);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_px) return;
    const int px = px_list[k];
    if (px < 0 || px >= F.npx) {
        pix[k].status = 2; pix[k].K = 0; pix[k].n_rec = 0; pix[k].n_can_open = 0;
        pix[k].A = pix[k].r = pix[k].phi = pix[k].out = 0.0f;
        return;
    }
    trace_pixel(P, T, F, px, pix + k, recs + (size_t)k * cap, cap);
}

// Kernel variant of a material (see shade_warp).
int kernel_variant(const KParams& P) {
    if (P.sampler) return kClassicalSampler;
    if (P.rng_table) return kRngTable;
    return P.M == 0 ? kIsoGrid : kRing;
}

static const void* fwd_kernel_fn(int v, bool two_d) {
    switch (v) {
        case kIsoGrid: return two_d ? reinterpret_cast<const void*>(&fwd_kernel<kIsoGrid, true>)
                                    : reinterpret_cast<const void*>(&fwd_kernel<kIsoGrid, false>);
        case kClassicalSampler: return two_d ? reinterpret_cast<const void*>(&fwd_kernel<kClassicalSampler, true>)
                                             : reinterpret_cast<const void*>(&fwd_kernel<kClassicalSampler, false>);
        case kRngTable: return two_d ? reinterpret_cast<const void*>(&fwd_kernel<kRngTable, true>)
                                     : reinterpret_cast<const void*>(&fwd_kernel<kRngTable, false>);
        default: return two_d ? reinterpret_cast<const void*>(&fwd_kernel<kRing, true>)
                              : reinterpret_cast<const void*>(&fwd_kernel<kRing, false>);
    }
}

const void* batch_kernel_fn(int v) {
    switch (v) {
        case kIsoGrid: return reinterpret_cast<const void*>(&batch_kernel<kIsoGrid>);
        case kClassicalSampler: return reinterpret_cast<const void*>(&batch_kernel<kClassicalSampler>);
        case kRngTable: return reinterpret_cast<const void*>(&batch_kernel<kRngTable>);
        default: return reinterpret_cast<const void*>(&batch_kernel<kRing>);
    }
}

static cudaError_t configure_smem() {
    static thread_local int configured_for = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_for == dev) return cudaSuccess;
    const int mx = (int)fwd_smem_bytes(1024);
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < kNumVariants && e == cudaSuccess; ++v) {
        e = cudaFuncSetAttribute(fwd_kernel_fn(v, false), cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fwd_kernel_fn(v, true), cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel_fn(v), cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    }
    if (e == cudaSuccess) configured_for = dev;
    return e;
}

cudaError_t launch_fwd(const KParams& P, const FrameDesc& F0, cudaStream_t s, FwdLaunch cfg) {
    cudaError_t e = configure_smem();
    if (e == cudaSuccess && P.rng_table) e = ensure_rng_table(s);
    if (e != cudaSuccess) return e;
    FrameDesc F = F0;
    const int rows1d = (F.npx + cfg.threads - 1) / cfg.threads;
    const int nt = frame_tiles(F, cfg.threads);
    if (cfg.blocks >= rows1d) cfg.blocks = nt;            // one CTA per tile (else a persistent grid)
    const size_t sm = fwd_smem_bytes(cfg.threads);
    switch (kernel_variant(P)) {
        case kIsoGrid:
            if (F.tile_w) fwd_kernel<kIsoGrid, true><<<cfg.blocks, cfg.threads, sm, s>>>(P, F);
            else fwd_kernel<kIsoGrid, false><<<cfg.blocks, cfg.threads, sm, s>>>(P, F);
            break;
        case kClassicalSampler:
            if (F.tile_w) fwd_kernel<kClassicalSampler, true><<<cfg.blocks, cfg.threads, sm, s>>>(P, F);
            else fwd_kernel<kClassicalSampler, false><<<cfg.blocks, cfg.threads, sm, s>>>(P, F);
            break;
        case kRngTable:
            if (F.tile_w) fwd_kernel<kRngTable, true><<<cfg.blocks, cfg.threads, sm, s>>>(P, F);
            else fwd_kernel<kRngTable, false><<<cfg.blocks, cfg.threads, sm, s>>>(P, F);
            break;
        default:
            if (F.tile_w) fwd_kernel<kRing, true><<<cfg.blocks, cfg.threads, sm, s>>>(P, F);
            else fwd_kernel<kRing, false><<<cfg.blocks, cfg.threads, sm, s>>>(P, F);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch(const KParams& P, const BatchDesc& B, cudaStream_t s, FwdLaunch cfg) {
    cudaError_t e = configure_smem();
    if (e == cudaSuccess && P.rng_table) e = ensure_rng_table(s);
    if (e != cudaSuccess) return e;
    const size_t sm = fwd_smem_bytes(cfg.threads);
    switch (kernel_variant(P)) {
        case kIsoGrid: batch_kernel<kIsoGrid><<<cfg.blocks, cfg.threads, sm, s>>>(P, B); break;
        case kClassicalSampler: batch_kernel<kClassicalSampler><<<cfg.blocks, cfg.threads, sm, s>>>(P, B); break;
        case kRngTable: batch_kernel<kRngTable><<<cfg.blocks, cfg.threads, sm, s>>>(P, B); break;
        default: batch_kernel<kRing><<<cfg.blocks, cfg.threads, sm, s>>>(P, B); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_trace(const KParams& P, const FrameDesc& F, const int32_t* px, int32_t n_px,
                         GlintTracePix* pix, GlintTraceRec* recs, int32_t cap, cudaStream_t s) {
    if (P.rng_table) {
        const cudaError_t e = ensure_rng_table(s);
        if (e != cudaSuccess) return e;
    }
    const int threads = 128;
    const int blocks = (n_px + threads - 1) / threads;
    trace_kernel<<<blocks, threads, 0, s>>>(P, F, px, n_px, pix, recs, cap);
    return cudaGetLastError();
}

}  // namespace glint
