// Plain forward kernel (one frame) and the parity-trace kernel.
#include "glint_kernels.cuh"

namespace glint {

// Copy the double-float tables (only the rotation entries up to ring M)
// from the parameter block into shared memory.
__device__ __forceinline__ void load_tables(const KParams& P, Tables& T) {
    const int nwords = (int)(sizeof(DfTables) / 4) + rot_entries(P.M) * (int)(sizeof(RotEntry) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&P.tables);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&T);
    for (int k = threadIdx.x; k < nwords; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

template <int NLT>
__global__ void __launch_bounds__(256) fwd_kernel(const __grid_constant__ KParams P) {
    __shared__ Tables T;
    load_tables(P, T);
    const int stride = gridDim.x * blockDim.x;
    for (int px = blockIdx.x * blockDim.x + threadIdx.x; px < P.npx; px += stride) {
        NoSink s;
        P.out[px] = shade_pixel<NLT>(P, T, px, s);
    }
}

struct TraceSink {
    static constexpr bool kTrace = true;
    GlintTracePix* pixrec;
    GlintTraceRec* recs;
    int cap;
    int nmax;
    __device__ void pix(int status, int K, float A, float r, float phi, float out) {
        pixrec->status = status; pixrec->K = K; pixrec->A = A; pixrec->r = r; pixrec->phi = phi;
        pixrec->out = out; pixrec->n_rec = nmax; pixrec->pad = 0;
    }
    __device__ void rec(int idx, int light, int sub, int vert, int sv, int av, uint32_t gid, int i, int j,
                        int ax, int ay, uint32_t h0, uint32_t h1, int gate, int c, float n, float P1,
                        float mu, float sigma, float cc, float u, float v, float p) {
        nmax = idx + 1 > nmax ? idx + 1 : nmax;
        pixrec->n_rec = nmax;
        if (idx >= cap) return;
        GlintTraceRec& R = recs[idx];
        R.light = light; R.sub = sub; R.vert = vert; R.sv = sv; R.av = av; R.grid_id = gid;
        R.i = i; R.j = j; R.ax = ax; R.ay = ay; R.h0 = h0; R.h1 = h1; R.gate = gate; R.c = c;
        R.n = n; R.P1 = P1; R.mu = mu; R.sigma = sigma; R.c_cont = cc; R.u = u; R.v = v; R.p = p;
    }
};

__global__ void __launch_bounds__(128) trace_kernel(const __grid_constant__ KParams P, const int32_t* px_list,
                                                    int32_t n_px, GlintTracePix* pix, GlintTraceRec* recs,
                                                    int32_t cap) {
    __shared__ Tables T;
    load_tables(P, T);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_px) return;
    const int px = px_list[k];
    TraceSink s{pix + k, recs + (size_t)k * cap, cap, 0};
    if (px < 0 || px >= P.npx) { s.pix(2, 0, 0.f, 0.f, 0.f, 0.f); return; }
    shade_pixel<0>(P, T, px, s);
}

cudaError_t launch_fwd(const KParams& P, cudaStream_t s, FwdLaunch cfg) {
    if (P.nL == 1) fwd_kernel<1><<<cfg.blocks, cfg.threads, 0, s>>>(P);
    else if (P.nL == 2) fwd_kernel<2><<<cfg.blocks, cfg.threads, 0, s>>>(P);
    else fwd_kernel<0><<<cfg.blocks, cfg.threads, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_trace(const KParams& P, const int32_t* px, int32_t n_px, GlintTracePix* pix,
                         GlintTraceRec* recs, int32_t cap, cudaStream_t s) {
    const int threads = 128;
    const int blocks = (n_px + threads - 1) / threads;
    trace_kernel<<<blocks, threads, 0, s>>>(P, px, n_px, pix, recs, cap);
    return cudaGetLastError();
}

}  // namespace glint
