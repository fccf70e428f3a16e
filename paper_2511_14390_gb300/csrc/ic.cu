// Direct-form initial conditions: past inputs x[-1..-N] and past outputs y[-1..-M] (the
// convention of SciPy's lfiltic and MATLAB's filtic) turned into the TDF-II state the
// filter entry points take, and the adjoint of that map.  Sec. 2 pairs the direct form
// with its transposed form; the TDF-II state at n = 0 is what the past terms of the
// difference equation (Eq. rtf) add to the first M outputs:
//     zi[m] = sum_{k=m+1..N} b_k x[m-k] - sum_{k=m+1..M} a_k y[m-k],   m = 0..M-1
// Linear in the past values and in the coefficients, so its adjoint, given
// gzi = dL/dzi from the filter's backward, is
//     dL/dx[-j] = sum_m gzi[m] b_{m+j},   dL/dy[-j] = -sum_m gzi[m] a_{m+j}
//     dL/db_k  += sum_{m<k} gzi[m] x[m-k],   dL/da_k += -sum_{m<k} gzi[m] y[m-k]
// (the second line completes the filter's own coefficient gradients with the terms
// of the past values).  Both are tiny: one thread per state entry or per output.
#include "kernels.h"

using namespace dfilt;

namespace {

__global__ void ic_df1_kernel(const float *__restrict__ b, const float *__restrict__ a,
                              const float *__restrict__ xp, const float *__restrict__ yp,
                              float *__restrict__ zi, int64_t B, int N, int M) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= B * M) return;
    const int64_t ch = id / M;
    const int m = (int)(id - ch * M);
    float acc = 0.0f;
    if (xp)
        for (int k = m + 1; k <= N; ++k) acc = fmaf(b[ch * (N + 1) + k], xp[ch * N + (k - m - 1)], acc);
    if (yp)
        for (int k = m + 1; k <= M; ++k) acc = fmaf(-a[ch * M + k - 1], yp[ch * M + (k - m - 1)], acc);
    zi[id] = acc;
}

// One block of 64 threads per channel; thread t forms entry t of each output.
__global__ void __launch_bounds__(64)
ic_df1_bwd_kernel(const float *__restrict__ b, const float *__restrict__ a,
                  const float *__restrict__ xp, const float *__restrict__ yp,
                  const float *__restrict__ gzi, float *__restrict__ gxp,
                  float *__restrict__ gyp, float *__restrict__ gb, float *__restrict__ ga,
                  int N, int M) {
    const int64_t ch = blockIdx.x;
    const int t = threadIdx.x;
    const float *g = gzi + ch * M;
    const int j = t + 1;                           // lag of the past value
    if (gxp && j <= N) {
        float acc = 0.0f;
        for (int m = 0; m < M && m + j <= N; ++m) acc = fmaf(g[m], b[ch * (N + 1) + m + j], acc);
        gxp[ch * N + t] = acc;
    }
    if (gyp && j <= M) {
        float acc = 0.0f;
        for (int m = 0; m + j <= M; ++m) acc = fmaf(g[m], a[ch * M + m + j - 1], acc);
        gyp[ch * M + t] = -acc;
    }
    if (gb && xp && j <= N) {                      // k = j: terms m < k, x[m-k] = xp[k-m-1]
        float acc = 0.0f;
        for (int m = 0; m < j && m < M; ++m) acc = fmaf(g[m], xp[ch * N + (j - m - 1)], acc);
        gb[ch * (N + 1) + j] += acc;
    }
    if (ga && yp && j <= M) {
        float acc = 0.0f;
        for (int m = 0; m < j; ++m) acc = fmaf(g[m], yp[ch * M + (j - m - 1)], acc);
        ga[ch * M + j - 1] -= acc;
    }
}

}  // namespace

extern "C" dfilt_status dfilt_ic_df1(const float *b, const float *a, const float *xpast,
                                     const float *ypast, float *zi, int64_t B, int N, int M,
                                     void *stream) {
    if (B < 0) return DFILT_ERR_INVALID_ARG;
    if (M > 64) return DFILT_ERR_UNSUPPORTED;
    if (M < 1 || N < 0 || N > M) return DFILT_ERR_INVALID_ARG;
    if (B == 0) return DFILT_OK;
    if (!zi || (xpast && N > 0 && !b) || (ypast && !a)) return DFILT_ERR_INVALID_ARG;
    const int64_t n = B * M;
    ic_df1_kernel<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        b, a, N > 0 ? xpast : nullptr, ypast, zi, B, N, M); note_launch();
    return cudaGetLastError() == cudaSuccess ? DFILT_OK : DFILT_ERR_CUDA;
}

extern "C" dfilt_status dfilt_ic_df1_backward(const float *b, const float *a, const float *xpast,
                                              const float *ypast, const float *gzi,
                                              float *gxpast, float *gypast, float *gb,
                                              float *ga, int64_t B, int N, int M,
                                              void *stream) {
    if (B < 0) return DFILT_ERR_INVALID_ARG;
    if (M > 64) return DFILT_ERR_UNSUPPORTED;
    if (M < 1 || N < 0 || N > M) return DFILT_ERR_INVALID_ARG;
    if (B == 0) return DFILT_OK;
    if (!gzi || ((gxpast || gb) && N > 0 && !b) || ((gypast || ga) && !a)) return DFILT_ERR_INVALID_ARG;
    if (B > 0x7fffffffLL) return DFILT_ERR_UNSUPPORTED;
    ic_df1_bwd_kernel<<<(unsigned)B, 64, 0, static_cast<cudaStream_t>(stream)>>>(
        b, a, N > 0 ? xpast : nullptr, ypast, gzi, N > 0 ? gxpast : nullptr, gypast, gb, ga, N,
        M); note_launch();
    return cudaGetLastError() == cudaSuccess ? DFILT_OK : DFILT_ERR_CUDA;
}
