// dfilt_jvp: forward-mode derivative (Jacobian-vector product) of the filter.
//
// The forward is linear in the signal for fixed coefficients: A(z) y = B(z) x plus the
// initial state injected into the all-pole input.  Differentiating that identity along
// tangents (dx, db, da, dzi) gives dA y + A dy = dB x + B dx + (dzi injected), so
//
//     v[n]  = sum_{k=0..N} (b_k dx[n-k] + db_k x[n-k]) - sum_{k=1..M} da_k y[n-k]
//     dy    = 1/A applied to v, TDF-II initial state dzi
//
// (causal sums: x, dx, y are zero at negative times; y is the forward's output, which
// already carries the zi response).  This is the forward-mode counterpart of the
// reverse-mode gradients of Sec. 3.1, which Sec. 5 notes follows the same way.  The
// call runs two steps: `jvp_input_kernel` (or its low-order streaming form) forms v (a
// short FIR over three signals, HBM-bound: 12 bytes read and 4 written per sample), then the library's own forward
// filters v with numerator [1] and state dzi, so the recursion runs on the chunked
// tensor-core path (or the sequential kernel, as opts select).
#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

using namespace dfilt;

namespace {

constexpr int kJvpThreads = 256;
constexpr int kJvpPer = 8;                               // outputs per thread
constexpr int kJvpSeg = kJvpThreads * kJvpPer;           // samples per block
constexpr int kJvpHalo = 64;                             // max(N, M) <= 64
constexpr int kJvpLoads = (kJvpSeg + kJvpHalo + kJvpThreads - 1) / kJvpThreads;

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

// One block per (channel, segment of kJvpSeg samples): the segment and its halo of
// the needed signals are staged in shared memory with coalesced loads (all loads of a
// thread issued before any is stored), then every thread forms kJvpPer outputs
// spaced kJvpThreads apart (conflict-free shared-memory reads).  Block 0.. also
// write ones[i] = 1 for i < B (the numerator [1] of the second step).
__global__ void __launch_bounds__(kJvpThreads)
jvp_input_kernel(const float *__restrict__ x, const float *__restrict__ dx,
                 const float *__restrict__ y, const float *__restrict__ b,
                 const float *__restrict__ db, const float *__restrict__ da,
                 float *__restrict__ v, float *__restrict__ ones, int64_t B, int64_t T, int N,
                 int M, int64_t segs) {
    __shared__ float xs[kJvpSeg + kJvpHalo], dxs[kJvpSeg + kJvpHalo], ys[kJvpSeg + kJvpHalo];
    __shared__ float cb[kJvpHalo + 1], cdb[kJvpHalo + 1], cda[kJvpHalo + 1];
    const int tid = threadIdx.x;
    const int64_t gid = (int64_t)blockIdx.x * kJvpThreads + tid;
    if (gid < B) ones[gid] = 1.0f;

    const int64_t ch = (int64_t)blockIdx.x / segs;
    const int64_t n0 = ((int64_t)blockIdx.x - ch * segs) * kJvpSeg;
    const int64_t n1 = n0 + kJvpSeg < T ? n0 + kJvpSeg : T;
    const int H = N > M ? N : M;
    const int cnt = (int)(n1 - n0) + H;                  // staged samples n0-H .. n1-1
    const int64_t row = ch * T;
    const bool use_dx = dx != nullptr, use_db = db != nullptr, use_da = da != nullptr;

    if (tid <= N) {
        cb[tid] = use_dx ? b[ch * (N + 1) + tid] : 0.0f;
        cdb[tid] = use_db ? db[ch * (N + 1) + tid] : 0.0f;
    }
    if (tid < M) cda[tid + 1] = use_da ? da[ch * M + tid] : 0.0f;

    float rx[kJvpLoads], rdx[kJvpLoads], ry[kJvpLoads];
#pragma unroll
    for (int r = 0; r < kJvpLoads; ++r) {
        const int idx = tid + r * kJvpThreads;
        const int64_t n = n0 - H + idx;
        const bool in = idx < cnt && n >= 0;
        rx[r] = (in && use_db) ? __ldcs(x + row + n) : 0.0f;
        rdx[r] = (in && use_dx) ? __ldcs(dx + row + n) : 0.0f;
        ry[r] = (in && use_da) ? __ldcs(y + row + n) : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < kJvpLoads; ++r) {
        const int idx = tid + r * kJvpThreads;
        if (idx < cnt) {
            xs[idx] = rx[r];
            dxs[idx] = rdx[r];
            ys[idx] = ry[r];
        }
    }
    __syncthreads();

#pragma unroll
    for (int j = 0; j < kJvpPer; ++j) {
        const int t = tid + j * kJvpThreads;
        if (n0 + t < n1) {
            const int c = t + H;                         // staged index of sample n0 + t
            float acc = 0.0f;
            for (int k = 0; k <= N; ++k) acc = fmaf(cb[k], dxs[c - k], fmaf(cdb[k], xs[c - k], acc));
            for (int k = 1; k <= M; ++k) acc = fmaf(-cda[k], ys[c - k], acc);
            v[row + n0 + t] = acc;
        }
    }
}

// Low orders (max(N, M) <= 4) on rows of a multiple of 4 samples with 16-byte aligned
// signals: a streaming kernel without shared memory.  Grid x covers the quads of a row,
// grid y strides over rows; thread q forms the 4 outputs of quad q of its row from one
// float4 load per signal, and the quad before it (the window's history) comes from the
// neighbouring lane by shuffle (lane 0 loads it; it is zero at a row's start).  Same
// terms in the same order as jvp_input_kernel.  Lanes past a row's end mirror its last
// quad and store nothing, so the shuffles always run with the full warp.
__device__ __forceinline__ float4 shfl_up4(float4 a) {
    a.x = __shfl_up_sync(0xffffffffu, a.x, 1);
    a.y = __shfl_up_sync(0xffffffffu, a.y, 1);
    a.z = __shfl_up_sync(0xffffffffu, a.z, 1);
    a.w = __shfl_up_sync(0xffffffffu, a.w, 1);
    return a;
}

template <int H>   // max(N, M): the history each output needs
__global__ void __launch_bounds__(kJvpThreads, H <= 2 ? 6 : 4)
jvp_input_vec4_kernel(const float4 *__restrict__ x, const float4 *__restrict__ dx,
                      const float4 *__restrict__ y, const float *__restrict__ b,
                      const float *__restrict__ db, const float *__restrict__ da,
                      float4 *__restrict__ v, float *__restrict__ ones, int64_t B, int64_t T,
                      int N, int M) {
    const int64_t nqr = T / 4;                           // quads per row
    const int64_t qr = (int64_t)blockIdx.x * kJvpThreads + threadIdx.x;
    const bool live = qr < nqr;
    const int64_t qc = live ? qr : nqr - 1;
    const int lane = threadIdx.x & 31;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    __shared__ float cb[H + 1], cdb[H + 1], cda[H + 1];
    for (int64_t row = blockIdx.y; row < B; row += gridDim.y) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ones[row] = 1.0f;
        const int64_t qq = row * nqr + qc;
        __syncthreads();                                 // previous row's coefficients read
        if (threadIdx.x <= H) {
            const int k = threadIdx.x;
            cb[k] = (dx && k <= N) ? __ldg(b + row * (N + 1) + k) : 0.0f;
            cdb[k] = (db && k <= N) ? __ldg(db + row * (N + 1) + k) : 0.0f;
            cda[k] = (da && k >= 1 && k <= M) ? __ldg(da + row * M + k - 1) : 0.0f;
        }
        const float4 cx = db ? __ldcs(x + qq) : z4;
        const float4 cdx = dx ? __ldcs(dx + qq) : z4;
        const float4 cy = da ? __ldcs(y + qq) : z4;
        float4 px = shfl_up4(cx), pdx = shfl_up4(cdx), py = shfl_up4(cy);
        if (qc == 0) {
            px = pdx = py = z4;
        } else if (lane == 0) {
            px = db ? __ldg(x + qq - 1) : z4;
            pdx = dx ? __ldg(dx + qq - 1) : z4;
            py = da ? __ldg(y + qq - 1) : z4;
        }
        __syncthreads();                                 // this row's coefficients written
        const float xw[8] = {px.x, px.y, px.z, px.w, cx.x, cx.y, cx.z, cx.w};
        const float dxw[8] = {pdx.x, pdx.y, pdx.z, pdx.w, cdx.x, cdx.y, cdx.z, cdx.w};
        const float yw[8] = {py.x, py.y, py.z, py.w, cy.x, cy.y, cy.z, cy.w};
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 4 + j;
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k <= H; ++k)
                if (k <= N) acc = fmaf(cb[k], dxw[c - k], fmaf(cdb[k], xw[c - k], acc));
#pragma unroll
            for (int k = 1; k <= H; ++k)
                if (k <= M) acc = fmaf(-cda[k], yw[c - k], acc);
            o[j] = acc;
        }
        if (live) v[qq] = make_float4(o[0], o[1], o[2], o[3]);
    }
}

bool aligned16p(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Workspace layout: v [B*T floats] | ones [B floats] | the forward's workspace.
struct JvpLayout {
    size_t v, ones, fwd, fwd_bytes, total;
};

dfilt_status jvp_layout(int64_t B, int64_t T, int M, const dfilt_opts *opts, JvpLayout *L) {
    size_t fws = 0;
    const dfilt_status s = dfilt_workspace_size(B, T, 0, M, opts, &fws, nullptr, nullptr);
    if (s != DFILT_OK) return s;
    L->v = 0;
    L->ones = align256((size_t)B * (size_t)T * sizeof(float));
    L->fwd = L->ones + align256((size_t)B * sizeof(float));
    L->fwd_bytes = fws;
    L->total = L->fwd + fws;
    return DFILT_OK;
}

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

}  // namespace

extern "C" dfilt_status dfilt_jvp_workspace_size(int64_t B, int64_t T, int N, int M,
                                                 const dfilt_opts *opts, size_t *ws_bytes) {
    if (B < 0 || T < 0) return DFILT_ERR_INVALID_ARG;
    if (M > 64) return DFILT_ERR_UNSUPPORTED;
    if (M < 1 || N < 0 || N > M) return DFILT_ERR_INVALID_ARG;
    JvpLayout L;
    const dfilt_status s = jvp_layout(B, T, M, opts, &L);
    if (s != DFILT_OK) return s;
    if (ws_bytes) *ws_bytes = L.total;
    return DFILT_OK;
}

extern "C" dfilt_status dfilt_jvp(const float *x, const float *y, const float *b, const float *a,
                                  const float *dx, const float *db, const float *da,
                                  const float *dzi, float *dy, void *ws, size_t ws_bytes,
                                  int64_t B, int64_t T, int N, int M, const dfilt_opts *opts,
                                  void *stream) {
    NvtxRange range("dfilt_jvp");
    if (B < 0 || T < 0) return DFILT_ERR_INVALID_ARG;
    if (M > 64) return DFILT_ERR_UNSUPPORTED;
    if (M < 1 || N < 0 || N > M) return DFILT_ERR_INVALID_ARG;
    JvpLayout L;
    const dfilt_status s = jvp_layout(B, T, M, opts, &L);
    if (s != DFILT_OK) return s;
    if (B == 0 || T == 0) return DFILT_OK;
    if (!a || !dy || (dx && !b) || (db && !x) || (da && !y)) return DFILT_ERR_INVALID_ARG;
    if (ws_bytes < L.total || !ws) return DFILT_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & 15) return DFILT_ERR_INVALID_ARG;
    char *w = static_cast<char *>(ws);
    float *v = reinterpret_cast<float *>(w + L.v);
    float *ones = reinterpret_cast<float *>(w + L.ones);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool vec4 = (N > M ? N : M) <= 4 && T % 4 == 0 && aligned16p(x) && aligned16p(dx) &&
                      aligned16p(y) && aligned16p(v);
    if (vec4) {
        const int64_t bx = (T / 4 + kJvpThreads - 1) / kJvpThreads;
        if (bx > 0x7fffffffLL) return DFILT_ERR_UNSUPPORTED;
        const dim3 grid((unsigned)bx, (unsigned)(B < 65535 ? B : 65535));
        auto *kern = jvp_input_vec4_kernel<4>;
        switch (N > M ? N : M) {
            case 1: kern = jvp_input_vec4_kernel<1>; break;
            case 2: kern = jvp_input_vec4_kernel<2>; break;
            case 3: kern = jvp_input_vec4_kernel<3>; break;
            default: break;
        }
        kern<<<grid, kJvpThreads, 0, st>>>(
            reinterpret_cast<const float4 *>(x), reinterpret_cast<const float4 *>(dx),
            reinterpret_cast<const float4 *>(y), b, db, da, reinterpret_cast<float4 *>(v), ones,
            B, T, N, M); note_launch();
    } else {
        const int64_t segs = (T + kJvpSeg - 1) / kJvpSeg;
        const int64_t blocks = B * segs;
        if (blocks > 0x7fffffffLL) return DFILT_ERR_UNSUPPORTED;
        jvp_input_kernel<<<(unsigned)blocks, kJvpThreads, 0, st>>>(x, dx, y, b, db, da, v, ones,
                                                                    B, T, N, M, segs); note_launch();
    }
    if (cudaGetLastError() != cudaSuccess) return DFILT_ERR_CUDA;
    return dfilt_forward(v, ones, a, dzi, dy, nullptr, w + L.fwd, L.fwd_bytes, B, T, 0, M, opts,
                         stream);
}
