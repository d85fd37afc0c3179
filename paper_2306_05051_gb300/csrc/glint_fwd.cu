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
#include "glint_kernels.cuh"

namespace glint {

constexpr int kQ = 64;                    // queue capacity per warp (ring)

struct WarpQueue {
    uint32_t word[kQ];                    // pre-image of the second hash word
    float mu[kQ], sig[kQ], nceil[kQ], w[kQ];
    int32_t owner[kQ];
    float res[32];
    uint32_t mask[32];
};

// Copy the double-float tables (only the rotation entries up to ring M)
// from the parameter block into shared memory.
__device__ __forceinline__ void load_tables(const KParams& P, Tables& T) {
    const int nwords = (int)(sizeof(DfTables) / 4) + rot_entries(P.M) * (int)(sizeof(RotEntry) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&P.tables);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&T);
    for (int k = threadIdx.x; k < nwords; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// Evaluate the n <= 32 queue entries starting at `head`: lane k takes entry
// head + k.  Each owner lane then adds its entries' values in queue order.
__device__ __noinline__ void flush_queue(WarpQueue& q, int head, int n, float& acc) {
    const int lane = threadIdx.x & 31;
    const int e = (head + lane) & (kQ - 1);
    float val = 0.0f;
    int owner = 32 + lane;                       // unique dummy for empty slots
    if (lane < n) {
        float cc;
        val = q.w[e] * open_count(fmix32(q.word[e]), q.mu[e], q.sig[e], q.nceil[e], &cc);
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
}

struct LightEval {          // what the evaluation loop needs of one light
    bool on;
    float p, lq, shade;
    float v[4];
    uint32_t A0[4], A1[4];
};

// Shade the pixel of this lane (px valid or not); all 32 lanes call together.
// ss0 / suw: the CTA's shared arrays of 12 x blockDim spatial words / weights.
// kIso: isotropic-grid mode (M = 0), tetrahedron vertices 0 and 3 only.
template <bool kIso>
__device__ float shade_warp(const KParams& P, const Tables& T, const FrameDesc& F, WarpQueue& q, int px,
                            bool valid, uint32_t* ss0, float* suw) {
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    PixelSetup S;
    S.status = 1;
    S.K = 0;
    if (valid) setup_pixel<false>(P, T, F, px, S);
    LightState ls[kMaxLights];
    bool any_on = false;
    for (int l = 0; l < F.nL; ++l) {
        ls[l].on = false;
        if (S.status == 0) setup_light<false>(P, F, S, px, l, ls[l]);
        any_on |= ls[l].on;
    }
    // a pixel that no light reaches shades to 0: its sub-footprints are not set up
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
            in_range = setup_sub<false, kIso>(P, T, S, sub, U, s0s, uws, st);
            act = in_range;
        }
#pragma unroll 1
        for (int l = 0; l < F.nL; ++l) {
            LightEval L;
            L.on = act && ls[l].on;
            L.p = ls[l].p; L.lq = ls[l].lq; L.shade = ls[l].shade;
#pragma unroll
            for (int k = 0; k < 4; ++k) { L.v[k] = ls[l].v[k]; L.A0[k] = ls[l].A0[k]; L.A1[k] = ls[l].A1[k]; }
            if (!__any_sync(0xffffffffu, L.on)) continue;
#pragma unroll 1
            for (int ii = 0; ii < (kIso ? 2 : 4); ++ii) {
                const int i = kIso ? 3 * ii : ii;
                CountLaw law = count_law(S.ntr[i], L.p, L.lq);
                if (!L.on) law.Tg = 0u;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const uint32_t s0 = s0s[(3 * i + j) * st], s1 = U.S1[3 * i + j];
                    const float uw = uws[(3 * i + j) * st] * L.shade;
                    // one warp vote for the 4 angular texels: most groups have no open gate
                    bool gk[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) gk[k] = gate_open(fmix32(s0 + L.A0[k]), law.Tg);
                    if (!__any_sync(0xffffffffu, gk[0] | gk[1] | gk[2] | gk[3])) continue;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool g = gk[k];
                        const unsigned m = __ballot_sync(0xffffffffu, g);
                        if (m) {
                            if (g) {
                                const int pos = (head + count + __popc(m & lt_mask)) & (kQ - 1);
                                q.word[pos] = s1 + L.A1[k];
                                q.mu[pos] = law.mu; q.sig[pos] = law.sig; q.nceil[pos] = law.nceil;
                                q.w[pos] = uw * L.v[k];
                                q.owner[pos] = lane;
                            }
                            count += __popc(m);
                            if (count >= 32) {
                                __syncwarp();
                                flush_queue(q, head, 32, acc);
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
        flush_queue(q, head, count, acc);
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

template <bool kIso>
__global__ void __launch_bounds__(1024) fwd_kernel(const __grid_constant__ KParams P, const FrameDesc F) {
    extern __shared__ __align__(16) unsigned char smem[];
    Tables& T = *reinterpret_cast<Tables*>(smem);
    WarpQueue* Qs = reinterpret_cast<WarpQueue*>(smem + sizeof(Tables));
    uint32_t* ss0 = reinterpret_cast<uint32_t*>(Qs + blockDim.x / 32);
    float* suw = reinterpret_cast<float*>(ss0 + 12 * blockDim.x);
    load_tables(P, T);
    WarpQueue& q = Qs[threadIdx.x >> 5];
    // Block-uniform tiles of blockDim.x pixels.  The barrier at the top of a
    // tile keeps the block's warps together in the (long, mostly
    // straight-line) setup code so they share instruction-cache lines.
    for (int base = blockIdx.x * blockDim.x; base < F.npx; base += gridDim.x * blockDim.x) {
        __syncthreads();
        const int px = base + tile_pixel();
        const float o = shade_warp<kIso>(P, T, F, q, px, px < F.npx, ss0, suw);
        if (px < F.npx) __stcs(F.out + px, o);
    }
}

// Kernel over the tiles of many frames; tile t belongs to frame f with
// tile_base[f] <= t < tile_base[f+1].  Persistent: CTAs take tiles from a
// global counter (reset to 0 before the launch).  Otherwise one CTA per tile
// (CTA b shades tile b), scheduled by the hardware.
template <bool kIso>
__global__ void __launch_bounds__(1024) batch_kernel(const __grid_constant__ KParams P,
                                                     const __grid_constant__ BatchDesc B) {
    extern __shared__ __align__(16) unsigned char smem[];
    Tables& T = *reinterpret_cast<Tables*>(smem);
    WarpQueue* Qs = reinterpret_cast<WarpQueue*>(smem + sizeof(Tables));
    uint32_t* ss0 = reinterpret_cast<uint32_t*>(Qs + blockDim.x / 32);
    float* suw = reinterpret_cast<float*>(ss0 + 12 * blockDim.x);
    __shared__ int tile_s;
    load_tables(P, T);
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
        const int px = (t - B.tile_base[lo]) * (int)blockDim.x + tile_pixel();
        const float o = shade_warp<kIso>(P, T, F, q, px, px < F.npx, ss0, suw);
        if (px < F.npx) __stcs(F.out + px, o);
    }
}

size_t fwd_smem_bytes(int threads) {
    return sizeof(Tables) + (size_t)(threads / 32) * sizeof(WarpQueue) + (size_t)threads * 24 * sizeof(uint32_t);
}

// --------------------------------------------------------------------------
// parity trace: one thread per listed pixel, every evaluation recorded
// --------------------------------------------------------------------------
__device__ void trace_pixel(const KParams& P, const Tables& T, const FrameDesc& F, int px, GlintTracePix* pr,
                            GlintTraceRec* recs, int cap) {
    PixelSetup S;
    setup_pixel<true>(P, T, F, px, S);
    pr->status = S.status; pr->K = S.status == 0 ? S.K : 0; pr->n_rec = 0; pr->pad = 0;
    pr->A = S.status == 0 ? S.A.hi : 0.0f; pr->r = S.status == 0 ? S.ratio.hi : 0.0f;
    pr->phi = S.status == 0 ? S.phi.hi : 0.0f; pr->out = 0.0f;
    if (S.status != 0) return;
    LightState ls[kMaxLights];
    for (int l = 0; l < F.nL; ++l) setup_light<true>(P, F, S, px, l, ls[l]);
    float C[kMaxLights];
    for (int l = 0; l < F.nL; ++l) C[l] = 0.0f;
    int nrec = 0;
    for (int sub = 0; sub < S.K; ++sub) {
        SubState U;
        const bool ok = P.M > 0 ? setup_sub<true, false>(P, T, S, sub, U, U.S0, U.uw, 1)
                                : setup_sub<true, true>(P, T, S, sub, U, U.S0, U.uw, 1);
        if (!ok) { pr->status = 3; pr->n_rec = nrec; return; }
        for (int l = 0; l < F.nL; ++l) {
            const LightState& L = ls[l];
            if (!L.on) continue;
            for (int i = 0; i < 4; ++i) {
                if (!vertex_used(P.M, i)) continue;
                const CountLaw law = count_law(S.ntr[i], L.p, L.lq);
                for (int j = 0; j < 3; ++j) {
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t h0 = fmix32(U.S0[3 * i + j] + L.A0[k]);
                        const uint32_t h1 = fmix32(U.S1[3 * i + j] + L.A1[k]);
                        const bool g = gate_open(h0, law.Tg);
                        float c = 0.0f, cc = 0.0f;
                        if (g) {
                            c = open_count(h1, law.mu, law.sig, law.nceil, &cc);
                            C[l] += U.uw[3 * i + j] * L.v[k] * c;
                        }
                        const int idx = (((l * S.K + sub) * 4 + i) * 3 + j) * 4 + k;
                        ++nrec;
                        if (idx < cap) {
                            GlintTraceRec& R = recs[idx];
                            R.light = l; R.sub = sub; R.vert = i; R.sv = j; R.av = k; R.grid_id = U.gid[i];
                            R.i = U.li[3 * i + j]; R.j = U.lj[3 * i + j]; R.ax = L.ax[k]; R.ay = L.ay[k];
                            R.h0 = h0; R.h1 = h1; R.gate = g ? 1 : 0;
                            R.c = c < 2147483647.0f ? (int)c : 2147483647;
                            R.n = S.ntr[i]; R.P1 = law.P1; R.mu = law.mu; R.sigma = law.sig; R.c_cont = cc;
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
        pix[k].status = 2; pix[k].K = 0; pix[k].n_rec = 0; pix[k].pad = 0;
        pix[k].A = pix[k].r = pix[k].phi = pix[k].out = 0.0f;
        return;
    }
    trace_pixel(P, T, F, px, pix + k, recs + (size_t)k * cap, cap);
}

static cudaError_t configure_smem() {
    static thread_local int configured_for = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_for == dev) return cudaSuccess;
    const int mx = (int)fwd_smem_bytes(1024);
    cudaError_t e = cudaFuncSetAttribute(fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) configured_for = dev;
    return e;
}

cudaError_t launch_fwd(const KParams& P, const FrameDesc& F, cudaStream_t s, FwdLaunch cfg) {
    const cudaError_t e = configure_smem();
    if (e != cudaSuccess) return e;
    if (P.M == 0) fwd_kernel<true><<<cfg.blocks, cfg.threads, fwd_smem_bytes(cfg.threads), s>>>(P, F);
    else fwd_kernel<false><<<cfg.blocks, cfg.threads, fwd_smem_bytes(cfg.threads), s>>>(P, F);
    return cudaGetLastError();
}

cudaError_t launch_batch(const KParams& P, const BatchDesc& B, cudaStream_t s, FwdLaunch cfg) {
    const cudaError_t e = configure_smem();
    if (e != cudaSuccess) return e;
    if (P.M == 0) batch_kernel<true><<<cfg.blocks, cfg.threads, fwd_smem_bytes(cfg.threads), s>>>(P, B);
    else batch_kernel<false><<<cfg.blocks, cfg.threads, fwd_smem_bytes(cfg.threads), s>>>(P, B);
    return cudaGetLastError();
}

const void* batch_kernel_fn(bool iso) {
    return iso ? reinterpret_cast<const void*>(&batch_kernel<true>) : reinterpret_cast<const void*>(&batch_kernel<false>);
}

cudaError_t launch_trace(const KParams& P, const FrameDesc& F, const int32_t* px, int32_t n_px,
                         GlintTracePix* pix, GlintTraceRec* recs, int32_t cap, cudaStream_t s) {
    const int threads = 128;
    const int blocks = (n_px + threads - 1) / threads;
    trace_kernel<<<blocks, threads, 0, s>>>(P, F, px, n_px, pix, recs, cap);
    return cudaGetLastError();
}

}  // namespace glint
