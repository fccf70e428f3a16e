// The general linear recurrence of App. B, v(n+1) = A v(n) + z(n), with a dense M x M
// matrix A per channel (the operator the paper benchmarks at M = 2, Sec. 4), and its
// backward, which App. A / Eq. dLdz states as the same recurrence run with A^T on the
// time-reversed upstream gradient from a zero state, followed by
// dL/dv(0) = A^T dL/dz(0) and dL/dA = sum_n dL/dz(n) v(n)^T  (Eq. dLdvBA; v(n) the
// state before step n: v0, v(1), ..., v(T-1)).
//
// Chunked scan on the CUDA cores (M <= 4: a handful of FMAs per step, HBM-bound):
//   * a warp owns a segment of kSsSeg = 1024 steps, staged in shared memory with
//     coalesced loads; lane j runs the recurrence over its 32-step chunk from a zero
//     state (end state e_j), and a warp shuffle scan with the powers A^(32 * 2^k)
//     turns the e_j into chunk-end states;
//   * pass 1 keeps only the segment's aggregate; a carry kernel scans the segments of
//     each channel (one warp per channel, shuffle scan with A^(1024 * 2^k), a serial
//     carry between groups of 32 segments) into every segment's entry state;
//   * pass 2 repeats the chunk pass with the entry state injected at lane 0, reruns
//     each chunk from its true entry state in place in shared memory, and stores v.
// The powers A^(2^k), k = 5..14, are formed per channel by squaring in FP64.  z is
// read twice and v written once (24 bytes per step at M = 2).  The backward runs the
// same kernels on A^T in reversed time (no initial state) to get dL/dz, then a
// reduction kernel forms dL/dA (FP32 sums over 128 steps, FP64 sums after that, in
// a fixed order) and dL/dv(0).
#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

using namespace dfilt;

namespace {

constexpr int kSsChunk = 32;                       // steps per lane
constexpr int kSsSeg = 32 * kSsChunk;              // steps per warp (segment)
constexpr int kSsWarps = 4;                        // segments per block
constexpr int kSsPow = 10;                         // A^(2^k), k = 5 .. 14
constexpr int kSsMaxM = 4;

size_t al256(size_t n) { return (n + 255) / 256 * 256; }

// y = P x for an M x M row-major matrix P held in shared or global memory.
template <int M>
__device__ __forceinline__ void matvec(const float *P, const float (&x)[M], float (&y)[M]) {
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < M; ++j) acc = fmaf(P[i * M + j], x[j], acc);
        y[i] = acc;
    }
}

template <int M>
__device__ __forceinline__ void shfl_up_vec(const float (&x)[M], float (&y)[M], int d) {
#pragma unroll
    for (int i = 0; i < M; ++i) y[i] = __shfl_up_sync(0xffffffffu, x[i], d);
}

// Powers A^(2^k), k = 5..14, of A (or A^T with trans), squared in FP64, per channel.
template <int M>
__global__ void ss_setup_kernel(const float *__restrict__ A, float *__restrict__ pw, int64_t B,
                                int trans) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double P[M][M], Q[M][M];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int j = 0; j < M; ++j)
            P[i][j] = (double)(trans ? A[b * M * M + j * M + i] : A[b * M * M + i * M + j]);
    for (int k = 1; k <= 14; ++k) {
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = 0; j < M; ++j) {
                double acc = 0.0;
#pragma unroll
                for (int l = 0; l < M; ++l) acc = fma(P[i][l], P[l][j], acc);
                Q[i][j] = acc;
            }
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = 0; j < M; ++j) P[i][j] = Q[i][j];
        if (k >= 5) {
            float *dst = pw + (b * kSsPow + (k - 5)) * M * M;
#pragma unroll
            for (int i = 0; i < M; ++i)
#pragma unroll
                for (int j = 0; j < M; ++j) dst[i * M + j] = (float)P[i][j];
        }
    }
}

// One pass over the segments (FINAL = false: segment aggregates; true: v).  REV runs
// logical step i at memory position T-1-i.  Block = kSsWarps segments of one channel.
template <int M, bool REV, bool FINAL>
__global__ void __launch_bounds__(32 * kSsWarps)
ss_seg_kernel(const float *__restrict__ A, int trans, const float *__restrict__ pw,
              const float *__restrict__ z, float *__restrict__ out,
              const float *__restrict__ seg_in, float *__restrict__ agg, int64_t B, int64_t T,
              int64_t G, int64_t groups) {
    constexpr int ROW = kSsChunk * M + 1;          // padded chunk row (conflict-free lanes)
    extern __shared__ float smem[];
    float *pws = smem;                             // A^(32 * 2^k), k = 0..4
    float *zs = smem + 5 * M * M + (threadIdx.x >> 5) * (32 * ROW);
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x / groups;
    const int64_t g = ((int64_t)blockIdx.x - b * groups) * kSsWarps + (threadIdx.x >> 5);

    for (int i = threadIdx.x; i < 5 * M * M; i += blockDim.x) pws[i] = pw[b * kSsPow * M * M + i];
    float a[M * M];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int j = 0; j < M; ++j)
            a[i * M + j] = trans ? A[b * M * M + j * M + i] : A[b * M * M + i * M + j];
    __syncthreads();
    if (g >= G) return;                            // whole warp leaves together

    const int cnt = (int)((T - g * kSsSeg) < kSsSeg ? (T - g * kSsSeg) : kSsSeg);
    // memory positions of the segment: [p0, p0 + cnt)
    const int64_t p0 = REV ? T - g * kSsSeg - cnt : g * kSsSeg;
    const float *zb = z + (b * T + p0) * M;
    auto slot = [&](int f) {                       // shared-memory slot of segment float f
        const int pr = f / M, m = f - pr * M;
        const int l = REV ? cnt - 1 - pr : pr;
        return (l >> 5) * ROW + (l & 31) * M + m;
    };
    // every segment starts on a 16-byte boundary when T*M is a multiple of 4
    const bool vec = ((T * M) & 3) == 0 && (reinterpret_cast<uintptr_t>(z) & 15) == 0;
    const int nf = cnt * M;
    int done = 0;
    if (vec) {
        constexpr int R = 8;                       // float4 loads in flight per lane
        const float4 *z4 = reinterpret_cast<const float4 *>(zb);
        const int n4 = nf >> 2;
        for (int q0 = 0; q0 < n4; q0 += 32 * R) {
            float4 r4[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int q = q0 + r * 32 + lane;
                r4[r] = q < n4 ? __ldcs(z4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int q = q0 + r * 32 + lane;
                if (q < n4) {
                    zs[slot(4 * q)] = r4[r].x;
                    zs[slot(4 * q + 1)] = r4[r].y;
                    zs[slot(4 * q + 2)] = r4[r].z;
                    zs[slot(4 * q + 3)] = r4[r].w;
                }
            }
        }
        done = n4 * 4;
    }
    for (int f = done + lane; f < nf; f += 32) zs[slot(f)] = zb[f];
    __syncwarp();

    const int len = cnt - lane * kSsChunk < 0 ? 0 : (cnt - lane * kSsChunk > kSsChunk ? kSsChunk : cnt - lane * kSsChunk);
    float *zr = zs + lane * ROW;
    float s[M], t[M];
#pragma unroll
    for (int i = 0; i < M; ++i) s[i] = 0.0f;
    for (int st = 0; st < len; ++st) {
        matvec<M>(a, s, t);
#pragma unroll
        for (int i = 0; i < M; ++i) s[i] = t[i] + zr[st * M + i];
    }
    float e[M], sin_[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        e[i] = s[i];
        sin_[i] = 0.0f;
    }
    if (FINAL) {
#pragma unroll
        for (int i = 0; i < M; ++i) sin_[i] = seg_in[(b * G + g) * M + i];
        if (lane == 0) {
            matvec<M>(pws, sin_, t);               // A^32 times the segment's entry state
#pragma unroll
            for (int i = 0; i < M; ++i) e[i] += t[i];
        }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        float o[M];
        shfl_up_vec<M>(e, o, 1 << k);
        if (lane >= (1 << k)) {
            matvec<M>(pws + k * M * M, o, t);
#pragma unroll
            for (int i = 0; i < M; ++i) e[i] += t[i];
        }
    }
    if (!FINAL) {
        if (lane == 31) {
#pragma unroll
            for (int i = 0; i < M; ++i) agg[(b * G + g) * M + i] = e[i];
        }
        return;
    }
    float init[M];
    shfl_up_vec<M>(e, init, 1);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < M; ++i) init[i] = sin_[i];
    }
#pragma unroll
    for (int i = 0; i < M; ++i) s[i] = init[i];
    for (int st = 0; st < len; ++st) {
        matvec<M>(a, s, t);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            s[i] = t[i] + zr[st * M + i];
            zr[st * M + i] = s[i];
        }
    }
    __syncwarp();
    float *ob = out + (b * T + p0) * M;
    done = 0;
    if (vec && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        float4 *o4 = reinterpret_cast<float4 *>(ob);
        const int n4 = nf >> 2;
        for (int q = lane; q < n4; q += 32)
            o4[q] = make_float4(zs[slot(4 * q)], zs[slot(4 * q + 1)], zs[slot(4 * q + 2)],
                                zs[slot(4 * q + 3)]);
        done = n4 * 4;
    }
    for (int f = done + lane; f < nf; f += 32) ob[f] = zs[slot(f)];
}

// Entry state of every segment: one warp per channel, 32 segments at a time.
template <int M>
__global__ void __launch_bounds__(128)
ss_carry_kernel(const float *__restrict__ pw, const float *__restrict__ v0,
                const float *__restrict__ agg, float *__restrict__ seg_in, int64_t B, int64_t G) {
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (b >= B) return;
    const float *Q = pw + (b * kSsPow + 5) * M * M;  // A^(1024 * 2^k), k = 0..4
    float carry[M], t[M];
#pragma unroll
    for (int i = 0; i < M; ++i) carry[i] = v0 ? v0[b * M + i] : 0.0f;
    float nxt[M];                                  // aggregates of the next group, prefetched
#pragma unroll
    for (int i = 0; i < M; ++i) nxt[i] = lane < G ? agg[(b * G + lane) * M + i] : 0.0f;
    for (int64_t r = 0; r * 32 < G; ++r) {
        const int64_t g = r * 32 + lane;
        float e[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            e[i] = nxt[i];
            nxt[i] = g + 32 < G ? agg[(b * G + g + 32) * M + i] : 0.0f;
        }
        if (lane == 0) {
            matvec<M>(Q, carry, t);
#pragma unroll
            for (int i = 0; i < M; ++i) e[i] += t[i];
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            float o[M];
            shfl_up_vec<M>(e, o, 1 << k);
            if (lane >= (1 << k)) {
                matvec<M>(Q + k * M * M, o, t);
#pragma unroll
                for (int i = 0; i < M; ++i) e[i] += t[i];
            }
        }
        float init[M];
        shfl_up_vec<M>(e, init, 1);
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < M; ++i) init[i] = carry[i];
        }
        if (g < G) {
#pragma unroll
            for (int i = 0; i < M; ++i) seg_in[(b * G + g) * M + i] = init[i];
        }
#pragma unroll
        for (int i = 0; i < M; ++i) carry[i] = __shfl_sync(0xffffffffu, e[i], 31);
    }
}

// dL/dA partial sums per (channel, segment of kSsSeg steps): sum_n gz(n) prev(n)^T with
// prev(n) = v(n-1), prev(0) = v0.  Each thread sums its 4 steps in FP32, each warp
// its 128 steps by an FP32 shuffle tree (GB300's FP64 pipe is too narrow for a tree
// per warp), and the block adds the 8 warp sums in FP64 in a fixed order.
template <int M>
__global__ void __launch_bounds__(256)
ss_grada_kernel(const float *__restrict__ gz, const float *__restrict__ v,
                const float *__restrict__ v0, double *__restrict__ part, int64_t B, int64_t T,
                int64_t G) {
    __shared__ double red[8][M * M];
    const int64_t b = (int64_t)blockIdx.x / G;
    const int64_t g = (int64_t)blockIdx.x - b * G;
    float acc[M * M];
#pragma unroll
    for (int i = 0; i < M * M; ++i) acc[i] = 0.0f;
#pragma unroll
    for (int r = 0; r < kSsSeg / 256; ++r) {
        const int64_t n = g * kSsSeg + r * 256 + threadIdx.x;
        if (n < T) {
            float gv[M], pv[M];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                gv[i] = gz[(b * T + n) * M + i];
                pv[i] = n > 0 ? v[(b * T + n - 1) * M + i] : (v0 ? v0[b * M + i] : 0.0f);
            }
#pragma unroll
            for (int i = 0; i < M; ++i)
#pragma unroll
                for (int j = 0; j < M; ++j) acc[i * M + j] = fmaf(gv[i], pv[j], acc[i * M + j]);
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < M * M; ++i) {
        float d = acc[i];                          // FP32 tree over the warp's 128 steps
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        if (lane == 0) red[w][i] = (double)d;
    }
    __syncthreads();
    if (threadIdx.x < M * M) {
        double d = 0.0;
        for (int k = 0; k < 8; ++k) d += red[k][threadIdx.x];
        part[(b * G + g) * M * M + threadIdx.x] = d;
    }
}

// dL/dA = sum of the segment partials in order; dL/dv(0) = A^T dL/dz(0).
template <int M>
__global__ void ss_grada_final_kernel(const double *__restrict__ part, const float *__restrict__ A,
                                      const float *__restrict__ gz, float *__restrict__ gA,
                                      float *__restrict__ gv0, int64_t B, int64_t T, int64_t G) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= B * M * M) return;
    const int64_t b = id / (M * M);
    const int e = (int)(id - b * M * M);
    if (gA) {                                      // four interleaved chains, fixed order
        double d[4] = {0.0, 0.0, 0.0, 0.0};
        int64_t g = 0;
        for (; g + 4 <= G; g += 4)
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] += part[(b * G + g + k) * M * M + e];
        for (; g < G; ++g) d[0] += part[(b * G + g) * M * M + e];
        gA[id] = (float)((d[0] + d[1]) + (d[2] + d[3]));
    }
    if (gv0 && e < M) {                            // row e of A^T = column e of A
        float acc = 0.0f;
        if (T > 0)
            for (int j = 0; j < M; ++j) acc = fmaf(A[b * M * M + j * M + e], gz[b * T * M + j], acc);
        gv0[b * M + e] = acc;
    }
}

struct SsLayout {
    size_t pw, agg, seg_in, part, fwd_total, bwd_total;
    int64_t G;
};

SsLayout ss_layout(int64_t B, int64_t T, int M) {
    SsLayout L;
    L.G = (T + kSsSeg - 1) / kSsSeg;
    L.pw = 0;
    L.agg = L.pw + al256((size_t)B * kSsPow * M * M * sizeof(float));
    L.seg_in = L.agg + al256((size_t)B * L.G * M * sizeof(float));
    L.part = L.seg_in + al256((size_t)B * L.G * M * sizeof(float));
    L.fwd_total = L.part;
    L.bwd_total = L.part + al256((size_t)B * L.G * M * M * sizeof(double));
    return L;
}

template <int M, bool REV>
cudaError_t ss_scan(const float *A, int trans, const float *v0, const float *z, float *out,
                    char *ws, const SsLayout &L, int64_t B, int64_t T, cudaStream_t st) {
    float *pw = reinterpret_cast<float *>(ws + L.pw);
    float *agg = reinterpret_cast<float *>(ws + L.agg);
    float *seg_in = reinterpret_cast<float *>(ws + L.seg_in);
    ss_setup_kernel<M><<<(unsigned)((B + 127) / 128), 128, 0, st>>>(A, pw, B, trans); note_launch();
    if (L.G == 0) return cudaGetLastError();
    const int64_t groups = (L.G + kSsWarps - 1) / kSsWarps;
    const int64_t blocks = B * groups;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const size_t smem = (5 * M * M + kSsWarps * 32 * (kSsChunk * M + 1)) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(ss_seg_kernel<M, REV, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ss_seg_kernel<M, REV, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ss_seg_kernel<M, REV, false><<<(unsigned)blocks, 32 * kSsWarps, smem, st>>>(
        A, trans, pw, z, nullptr, nullptr, agg, B, T, L.G, groups); note_launch();
    ss_carry_kernel<M><<<(unsigned)((B + 3) / 4), 128, 0, st>>>(pw, v0, agg, seg_in, B, L.G); note_launch();
    ss_seg_kernel<M, REV, true><<<(unsigned)blocks, 32 * kSsWarps, smem, st>>>(
        A, trans, pw, z, out, seg_in, agg, B, T, L.G, groups); note_launch();
    return cudaGetLastError();
}

template <int M>
cudaError_t ss_forward_m(const float *A, const float *v0, const float *z, float *v, char *ws,
                         const SsLayout &L, int64_t B, int64_t T, cudaStream_t st) {
    return ss_scan<M, false>(A, 0, v0, z, v, ws, L, B, T, st);
}

template <int M>
cudaError_t ss_backward_m(const float *A, const float *v0, const float *v, const float *gv,
                          float *gA, float *gv0, float *gz, char *ws, const SsLayout &L,
                          int64_t B, int64_t T, cudaStream_t st) {
    cudaError_t e = ss_scan<M, true>(A, 1, nullptr, gv, gz, ws, L, B, T, st);
    if (e != cudaSuccess) return e;
    double *part = reinterpret_cast<double *>(ws + L.part);
    if (gA) {
        const int64_t blocks = B * L.G;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        if (blocks > 0)
            ss_grada_kernel<M><<<(unsigned)blocks, 256, 0, st>>>(gz, v, v0, part, B, T, L.G); note_launch();
    }
    if (gA || gv0) {
        const int64_t n = B * M * M;
        ss_grada_final_kernel<M><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, A, gz, gA,
                                                                           gv0, B, T, L.G); note_launch();
    }
    return cudaGetLastError();
}

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

dfilt_status to_status(cudaError_t e) { return e == cudaSuccess ? DFILT_OK : DFILT_ERR_CUDA; }

}  // namespace

extern "C" dfilt_status dfilt_ss_workspace_size(int64_t B, int64_t T, int M, size_t *fwd_ws,
                                                size_t *bwd_ws) {
    if (B < 0 || T < 0 || M < 1) return DFILT_ERR_INVALID_ARG;
    if (M > kSsMaxM) return DFILT_ERR_UNSUPPORTED;
    const SsLayout L = ss_layout(B, T, M);
    if (fwd_ws) *fwd_ws = L.fwd_total;
    if (bwd_ws) *bwd_ws = L.bwd_total;
    return DFILT_OK;
}

extern "C" dfilt_status dfilt_ss_forward(const float *A, const float *v0, const float *z,
                                         float *v, void *ws, size_t ws_bytes, int64_t B,
                                         int64_t T, int M, void *stream) {
    NvtxRange range("dfilt_ss_forward");
    if (B < 0 || T < 0 || M < 1) return DFILT_ERR_INVALID_ARG;
    if (M > kSsMaxM) return DFILT_ERR_UNSUPPORTED;
    if (B == 0 || T == 0) return DFILT_OK;
    if (!A || !z || !v) return DFILT_ERR_INVALID_ARG;
    const SsLayout L = ss_layout(B, T, M);
    if (!ws || ws_bytes < L.fwd_total) return DFILT_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & 15) return DFILT_ERR_INVALID_ARG;
    char *w = static_cast<char *>(ws);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (M) {
        case 1: return to_status(ss_forward_m<1>(A, v0, z, v, w, L, B, T, st));
        case 2: return to_status(ss_forward_m<2>(A, v0, z, v, w, L, B, T, st));
        case 3: return to_status(ss_forward_m<3>(A, v0, z, v, w, L, B, T, st));
        default: return to_status(ss_forward_m<4>(A, v0, z, v, w, L, B, T, st));
    }
}

extern "C" dfilt_status dfilt_ss_backward(const float *A, const float *v0, const float *v,
                                          const float *gv, float *gA, float *gv0, float *gz,
                                          void *ws, size_t ws_bytes, int64_t B, int64_t T, int M,
                                          void *stream) {
    NvtxRange range("dfilt_ss_backward");
    if (B < 0 || T < 0 || M < 1) return DFILT_ERR_INVALID_ARG;
    if (M > kSsMaxM) return DFILT_ERR_UNSUPPORTED;
    if (B == 0) return DFILT_OK;
    if (!A || !gz || (T > 0 && !gv) || (gA && T > 0 && !v)) return DFILT_ERR_INVALID_ARG;
    const SsLayout L = ss_layout(B, T, M);
    if (!ws || ws_bytes < L.bwd_total) return DFILT_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & 15) return DFILT_ERR_INVALID_ARG;
    char *w = static_cast<char *>(ws);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (M) {
        case 1: return to_status(ss_backward_m<1>(A, v0, v, gv, gA, gv0, gz, w, L, B, T, st));
        case 2: return to_status(ss_backward_m<2>(A, v0, v, gv, gA, gv0, gz, w, L, B, T, st));
        case 3: return to_status(ss_backward_m<3>(A, v0, v, gv, gA, gv0, gz, w, L, B, T, st));
        default: return to_status(ss_backward_m<4>(A, v0, v, gv, gA, gv0, gz, w, L, B, T, st));
    }
}
