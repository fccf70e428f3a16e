// Parameter-varying direct form (Sec. 5 notes the derivation extends to it): each output
// sample n has its own coefficients b[n][0..N], a[n][0..M-1],
//     y[n] = sum_{k=0..N} b[n][k] x[n-k] - sum_{k=1..M} a[n][k-1] y[n-k],
// x[n < 0] = 0, y[-1-j] = ypast[j].  Backward, with each coefficient taken at the output
// it produced (the same steps as App. A's adjoint, the transition now varying per step):
//     u[n] = gy[n] - sum_{k=1..M} a[n+k][k-1] u[n+k],  u[n >= T] = 0
//     grad_x[n] = sum_k b[n+k][k] u[n+k],  grad_b[n][k] = u[n] x[n-k],
//     grad_a[n][k-1] = -u[n] y[n-k],  grad_ypast[j] = -sum_{k>j} a[k-1-j][k-1] u[k-1-j].
//
// Both recursions are the same time-varying all-pole recursion o[i] = w[i] - sum_k c_k[i]
// o[i-k] (forward: w the FIR part, c_k[i] = a[i][k-1]; adjoint in reversed time i =
// T-1-n: w = gy, c_k[i] = a[n+k][k-1]).  With the state s_i = (o[i-1], ..., o[i-M]) a step
// is s_{i+1} = C_i s_i + e_1 w[i] with the companion matrix C_i, and a run of steps is the
// pair (product of the C_i, zero-start end state), combined by the paper's associative
// operator (A, z) + (A', z') = (A' A, A' z + z') (Sec. 3.2), here with a different A per
// step.  Chunked scan on the CUDA cores (M <= 4, FP32):
//   * a warp owns a segment of 1024 steps (w staged in shared memory, coalesced); lane j
//     runs its 32 steps from a zero state and the identity (pair P_j, e_j), a warp
//     shuffle scan with the operator gives every chunk's pair from the segment start;
//   * pass 1 keeps the segment's pair; a carry kernel (one thread per channel) steps the
//     segment entry states S_{g+1} = P_g S_g + e_g from S_0 = ypast (forward) or 0;
//   * pass 2 reruns each chunk from its entry state and writes o with coalesced stores.
// The FIR part and the gradients are element-wise kernels.
#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

using namespace dfilt;

namespace {

constexpr int kTvChunk = 32;
constexpr int kTvSeg = 32 * kTvChunk;
constexpr int kTvWarps = 4;
constexpr int kTvMaxM = 4;

size_t al256(size_t n) { return (n + 255) / 256 * 256; }

struct TvArgs {
    const float *w;      // [B][T] input of the recursion (memory order)
    const float *a;      // [B][T][M] denominators per output sample
    float *out;          // [B][T] output (memory order)
    float *pagg;         // [B][G][M*M] segment transition products
    float *eagg;         // [B][G][M] segment zero-start end states
    const float *seg_in; // [B][G][M] segment entry states
    int64_t B, T, G, groups;
};

// Coefficient c_k (k = 1..M) of logical step i (time n = i, or T-1-i for the adjoint).
template <int M, bool ADJ>
__device__ __forceinline__ void coeffs(const TvArgs &d, int64_t b, int64_t i, float (&c)[M]) {
    if constexpr (!ADJ) {
        const float *ar = d.a + (b * d.T + i) * M;
#pragma unroll
        for (int k = 0; k < M; ++k) c[k] = __ldg(ar + k);
    } else {
        const int64_t n = d.T - 1 - i;
#pragma unroll
        for (int k = 1; k <= M; ++k)
            c[k - 1] = n + k < d.T ? __ldg(d.a + (b * d.T + n + k) * M + (k - 1)) : 0.f;
    }
}

// One pass over the segments (FINAL = false: segment pairs; true: outputs).
template <int M, bool ADJ, bool FINAL>
__global__ void __launch_bounds__(32 * kTvWarps) tv_seg_kernel(TvArgs d) {
    constexpr int ROW = kTvChunk + 1;
    __shared__ float wsm[kTvWarps][32 * ROW];
    float *ws = wsm[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x / d.groups;
    const int64_t g = ((int64_t)blockIdx.x - b * d.groups) * kTvWarps + (threadIdx.x >> 5);
    if (g >= d.G) return;                            // whole warp leaves together
    const int cnt = (int)((d.T - g * kTvSeg) < kTvSeg ? (d.T - g * kTvSeg) : kTvSeg);
    const int64_t p0 = ADJ ? d.T - g * kTvSeg - cnt : g * kTvSeg;   // memory positions [p0, p0+cnt)
    auto slot = [&](int f) {                        // memory offset f -> logical slot
        const int l = ADJ ? cnt - 1 - f : f;
        return (l >> 5) * ROW + (l & 31);
    };
    const float *wb = d.w + b * d.T + p0;
    for (int f = lane; f < cnt; f += 32) ws[slot(f)] = __ldg(wb + f);
    __syncwarp();

    const int n = cnt - 32 * lane < 0 ? 0 : (cnt - 32 * lane > kTvChunk ? kTvChunk : cnt - 32 * lane);
    const int64_t i0 = g * kTvSeg + 32 * lane;      // the lane's first logical step
    float *row = ws + lane * ROW;
    // the chunk's pair from a zero state and the identity: P (row-major), e
    float P[M * M], e[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
        e[r] = 0.f;
#pragma unroll
        for (int q = 0; q < M; ++q) P[r * M + q] = r == q ? 1.f : 0.f;
    }
#pragma unroll 2
    for (int s = 0; s < n; ++s) {
        float c[M];
        coeffs<M, ADJ>(d, b, i0 + s, c);
        // e <- C e + e_1 w;  P <- C P  (C: first row -c, then the shift)
        float o = row[s];
#pragma unroll
        for (int k = 0; k < M; ++k) o = fmaf(-c[k], e[k], o);
#pragma unroll
        for (int k = M - 1; k > 0; --k) e[k] = e[k - 1];
        e[0] = o;
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float top = 0.f;
#pragma unroll
            for (int k = 0; k < M; ++k) top = fmaf(-c[k], P[k * M + q], top);
#pragma unroll
            for (int k = M - 1; k > 0; --k) P[k * M + q] = P[(k - 1) * M + q];
            P[q] = top;
        }
    }
    // inclusive warp scan, earlier lanes first: (P, e) <- (P P_left, P e_left + e)
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        float Pl[M * M], el[M];
#pragma unroll
        for (int t = 0; t < M * M; ++t) Pl[t] = __shfl_up_sync(0xffffffffu, P[t], dd);
#pragma unroll
        for (int t = 0; t < M; ++t) el[t] = __shfl_up_sync(0xffffffffu, e[t], dd);
        if (lane >= dd) {
            float Pn[M * M], en[M];
#pragma unroll
            for (int r = 0; r < M; ++r) {
                float acc = e[r];
#pragma unroll
                for (int k = 0; k < M; ++k) acc = fmaf(P[r * M + k], el[k], acc);
                en[r] = acc;
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    float s2 = 0.f;
#pragma unroll
                    for (int k = 0; k < M; ++k) s2 = fmaf(P[r * M + k], Pl[k * M + q], s2);
                    Pn[r * M + q] = s2;
                }
            }
#pragma unroll
            for (int t = 0; t < M * M; ++t) P[t] = Pn[t];
#pragma unroll
            for (int t = 0; t < M; ++t) e[t] = en[t];
        }
    }
    if constexpr (!FINAL) {
        if (lane == 31) {
#pragma unroll
            for (int t = 0; t < M * M; ++t) d.pagg[(b * d.G + g) * M * M + t] = P[t];
#pragma unroll
            for (int t = 0; t < M; ++t) d.eagg[(b * d.G + g) * M + t] = e[t];
        }
        return;
    } else {
        // the chunk's entry: the lanes before it applied to the segment entry
        float Pl[M * M], el[M], S[M], st[M];
#pragma unroll
        for (int t = 0; t < M * M; ++t) Pl[t] = __shfl_up_sync(0xffffffffu, P[t], 1);
#pragma unroll
        for (int t = 0; t < M; ++t) el[t] = __shfl_up_sync(0xffffffffu, e[t], 1);
#pragma unroll
        for (int t = 0; t < M; ++t) S[t] = d.seg_in[(b * d.G + g) * M + t];
#pragma unroll
        for (int r = 0; r < M; ++r) {
            if (lane == 0) {
                st[r] = S[r];
            } else {
                float acc = el[r];
#pragma unroll
                for (int k = 0; k < M; ++k) acc = fmaf(Pl[r * M + k], S[k], acc);
                st[r] = acc;
            }
        }
#pragma unroll 2
        for (int s = 0; s < n; ++s) {
            float c[M];
            coeffs<M, ADJ>(d, b, i0 + s, c);
            float o = row[s];
#pragma unroll
            for (int k = 0; k < M; ++k) o = fmaf(-c[k], st[k], o);
#pragma unroll
            for (int k = M - 1; k > 0; --k) st[k] = st[k - 1];
            st[0] = o;
            row[s] = o;
        }
        __syncwarp();
        float *ob = d.out + b * d.T + p0;
        for (int f = lane; f < cnt; f += 32) ob[f] = ws[slot(f)];
    }
}

// Segment entry states: S_0 = ypast (forward; the state holds past outputs in order) or
// zero (adjoint), S_{g+1} = P_g S_g + e_g.
template <int M>
__global__ void tv_carry_kernel(TvArgs d, const float *__restrict__ s0, float *__restrict__ seg_in) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.B) return;
    float S[M];
#pragma unroll
    for (int k = 0; k < M; ++k) S[k] = s0 ? s0[b * M + k] : 0.f;
    for (int64_t g = 0; g < d.G; ++g) {
#pragma unroll
        for (int k = 0; k < M; ++k) seg_in[(b * d.G + g) * M + k] = S[k];
        const float *P = d.pagg + (b * d.G + g) * M * M;
        const float *e = d.eagg + (b * d.G + g) * M;
        float Sn[M];
#pragma unroll
        for (int r = 0; r < M; ++r) {
            float acc = e[r];
#pragma unroll
            for (int k = 0; k < M; ++k) acc = fmaf(P[r * M + k], S[k], acc);
            Sn[r] = acc;
        }
#pragma unroll
        for (int k = 0; k < M; ++k) S[k] = Sn[k];
    }
}

// The FIR part of the forward: w[n] = sum_k b[n][k] x[n-k] (x[n < 0] = 0).
__global__ void tv_fir_kernel(const float *__restrict__ x, const float *__restrict__ bc,
                              float *__restrict__ w, int64_t B, int64_t T, int N) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B * T; i += stride) {
        const int64_t n = i % T;
        const float *br = bc + i * (N + 1);
        float acc = 0.f;
        for (int k = 0; k <= N; ++k)
            if (n - k >= 0) acc = fmaf(__ldg(br + k), __ldg(x + i - k), acc);
        w[i] = acc;
    }
}

// Gradients from the adjoint u (element-wise):
//   grad_x[n] = sum_k b[n+k][k] u[n+k],  grad_b[n][k] = u[n] x[n-k],
//   grad_a[n][k-1] = -u[n] y[n-k] (past outputs before n = 0);  each output may be NULL.
__global__ void tv_grad_kernel(const float *__restrict__ u, const float *__restrict__ x,
                               const float *__restrict__ y, const float *__restrict__ bc,
                               const float *__restrict__ yp, float *__restrict__ gx,
                               float *__restrict__ gb, float *__restrict__ ga, int64_t B,
                               int64_t T, int N, int M) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B * T; i += stride) {
        const int64_t ch = i / T, n = i - ch * T;
        const float un = __ldg(u + i);
        if (gx) {
            float acc = 0.f;
            for (int k = 0; k <= N; ++k)
                if (n + k < T) acc = fmaf(__ldg(bc + (i + k) * (N + 1) + k), __ldg(u + i + k), acc);
            gx[i] = acc;
        }
        if (gb)
            for (int k = 0; k <= N; ++k) gb[i * (N + 1) + k] = n - k >= 0 ? un * __ldg(x + i - k) : 0.f;
        if (ga)
            for (int k = 1; k <= M; ++k) {
                const float yk = n - k >= 0 ? __ldg(y + i - k) : (yp ? __ldg(yp + ch * M + (k - n - 1)) : 0.f);
                ga[i * M + k - 1] = -un * yk;
            }
    }
}

// grad_ypast[j] = -sum_{k=j+1..M} a[k-1-j][k-1] u[k-1-j]  (one thread per channel and j)
__global__ void tv_gyp_kernel(const float *__restrict__ u, const float *__restrict__ a,
                              float *__restrict__ gyp, int64_t B, int64_t T, int M) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * M) return;
    const int64_t ch = i / M;
    const int j = (int)(i - ch * M);
    float acc = 0.f;
    for (int k = j + 1; k <= M; ++k) {
        const int64_t n = k - 1 - j;
        if (n < T) acc = fmaf(__ldg(a + (ch * T + n) * M + k - 1), __ldg(u + ch * T + n), acc);
    }
    gyp[i] = -acc;
}

struct TvLayout {
    int64_t G;
    size_t buf, pagg, eagg, seg, total;
};

TvLayout tv_layout(int64_t B, int64_t T, int M) {
    TvLayout L{};
    L.G = (T + kTvSeg - 1) / kTvSeg;
    size_t o = 0;
    L.buf = o;
    o += al256((size_t)B * T * 4);
    L.pagg = o;
    o += al256((size_t)B * L.G * M * M * 4);
    L.eagg = o;
    o += al256((size_t)B * L.G * M * 4);
    L.seg = o;
    o += al256((size_t)B * L.G * M * 4);
    L.total = o;
    return L;
}

int grid_of(int64_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256, cap = (int64_t)(sms > 0 ? sms : 1) * 16;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <int M, bool ADJ>
cudaError_t tv_scan(const float *w, const float *a, const float *s0, float *out, char *ws,
                    const TvLayout &L, int64_t B, int64_t T, cudaStream_t st) {
    TvArgs d{};
    d.w = w;
    d.a = a;
    d.out = out;
    d.pagg = reinterpret_cast<float *>(ws + L.pagg);
    d.eagg = reinterpret_cast<float *>(ws + L.eagg);
    float *seg_in = reinterpret_cast<float *>(ws + L.seg);
    d.seg_in = seg_in;
    d.B = B;
    d.T = T;
    d.G = L.G;
    d.groups = (L.G + kTvWarps - 1) / kTvWarps;
    const int64_t blocks = B * d.groups;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    tv_seg_kernel<M, ADJ, false><<<(unsigned)blocks, 32 * kTvWarps, 0, st>>>(d); note_launch();
    tv_carry_kernel<M><<<(unsigned)((B + 127) / 128), 128, 0, st>>>(d, s0, seg_in); note_launch();
    tv_seg_kernel<M, ADJ, true><<<(unsigned)blocks, 32 * kTvWarps, 0, st>>>(d); note_launch();
    return cudaGetLastError();
}

template <int M>
cudaError_t tv_forward_m(const float *x, const float *bc, const float *a, const float *yp, float *y,
                         int N, char *ws, const TvLayout &L, int64_t B, int64_t T, cudaStream_t st) {
    float *w = reinterpret_cast<float *>(ws + L.buf);
    tv_fir_kernel<<<grid_of(B * T), 256, 0, st>>>(x, bc, w, B, T, N); note_launch();
    return tv_scan<M, false>(w, a, yp, y, ws, L, B, T, st);
}

template <int M>
cudaError_t tv_backward_m(const float *gy, const float *x, const float *y, const float *bc,
                          const float *a, const float *yp, float *gx, float *gb, float *ga,
                          float *gyp, int N, char *ws, const TvLayout &L, int64_t B, int64_t T,
                          cudaStream_t st) {
    float *u = reinterpret_cast<float *>(ws + L.buf);
    cudaError_t e = tv_scan<M, true>(gy, a, nullptr, u, ws, L, B, T, st);
    if (e != cudaSuccess) return e;
    if (gx || gb || ga) {
        tv_grad_kernel<<<grid_of(B * T), 256, 0, st>>>(u, x, y, bc, yp, gx, gb, ga, B, T, N, M); note_launch();
    }
    if (gyp) {
        tv_gyp_kernel<<<(unsigned)((B * M + 127) / 128), 128, 0, st>>>(u, a, gyp, B, T, M); note_launch();
    }
    return cudaGetLastError();
}

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

dfilt_status to_status(cudaError_t e) { return e == cudaSuccess ? DFILT_OK : DFILT_ERR_CUDA; }

dfilt_status tv_check(int64_t B, int64_t T, int N, int M) {
    if (B < 0 || T < 0 || M < 1 || N < 0) return DFILT_ERR_INVALID_ARG;
    if (M > kTvMaxM) return DFILT_ERR_UNSUPPORTED;
    if (N > M) return DFILT_ERR_INVALID_ARG;
    return DFILT_OK;
}

}  // namespace

extern "C" dfilt_status dfilt_tv_workspace_size(int64_t B, int64_t T, int N, int M, size_t *ws) {
    const dfilt_status s = tv_check(B, T, N, M);
    if (s != DFILT_OK) return s;
    if (ws) *ws = tv_layout(B, T, M).total;
    return DFILT_OK;
}

extern "C" dfilt_status dfilt_tv_forward(const float *x, const float *b, const float *a,
                                         const float *ypast, float *y, void *ws, size_t ws_bytes,
                                         int64_t B, int64_t T, int N, int M, void *stream) {
    NvtxRange range("dfilt_tv_forward");
    const dfilt_status s = tv_check(B, T, N, M);
    if (s != DFILT_OK) return s;
    if (B == 0 || T == 0) return DFILT_OK;
    if (!x || !b || !a || !y) return DFILT_ERR_INVALID_ARG;
    const TvLayout L = tv_layout(B, T, M);
    if (!ws || ws_bytes < L.total) return DFILT_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & 15) return DFILT_ERR_INVALID_ARG;
    char *w = static_cast<char *>(ws);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (M) {
        case 1: return to_status(tv_forward_m<1>(x, b, a, ypast, y, N, w, L, B, T, st));
        case 2: return to_status(tv_forward_m<2>(x, b, a, ypast, y, N, w, L, B, T, st));
        case 3: return to_status(tv_forward_m<3>(x, b, a, ypast, y, N, w, L, B, T, st));
        default: return to_status(tv_forward_m<4>(x, b, a, ypast, y, N, w, L, B, T, st));
    }
}

extern "C" dfilt_status dfilt_tv_backward(const float *gy, const float *x, const float *y,
                                          const float *b, const float *a, const float *ypast,
                                          float *gx, float *gb, float *ga, float *gypast,
                                          void *ws, size_t ws_bytes, int64_t B, int64_t T, int N,
                                          int M, void *stream) {
    NvtxRange range("dfilt_tv_backward");
    const dfilt_status s = tv_check(B, T, N, M);
    if (s != DFILT_OK) return s;
    if (B == 0) return DFILT_OK;
    if (T == 0) {
        if (gypast) {
            const cudaError_t e = cudaMemsetAsync(gypast, 0, (size_t)B * M * 4, static_cast<cudaStream_t>(stream));
            if (e != cudaSuccess) return DFILT_ERR_CUDA;
        }
        return DFILT_OK;
    }
    if (!gy || !a || (gx && !b) || (gb && !x) || (ga && !y)) return DFILT_ERR_INVALID_ARG;
    const TvLayout L = tv_layout(B, T, M);
    if (!ws || ws_bytes < L.total) return DFILT_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & 15) return DFILT_ERR_INVALID_ARG;
    char *w = static_cast<char *>(ws);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (M) {
        case 1: return to_status(tv_backward_m<1>(gy, x, y, b, a, ypast, gx, gb, ga, gypast, N, w, L, B, T, st));
        case 2: return to_status(tv_backward_m<2>(gy, x, y, b, a, ypast, gx, gb, ga, gypast, N, w, L, B, T, st));
        case 3: return to_status(tv_backward_m<3>(gy, x, y, b, a, ypast, gx, gb, ga, gypast, N, w, L, B, T, st));
        default: return to_status(tv_backward_m<4>(gy, x, y, b, a, ypast, gx, gb, ga, gypast, N, w, L, B, T, st));
    }
}
