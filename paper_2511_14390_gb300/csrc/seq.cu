// Sequential per-channel kernels: the direct recursion of Eq. rtf (forward, TDF-II
// state, Sec. 2) and its reverse-time adjoint (Sec. 3.1), one thread per channel.
//
// A warp owns 32 channels.  Signals stream through shared memory in 32x32 tiles:
// the warp reads a tile with coalesced row loads (next tile prefetched into
// registers while the current one is filtered), each lane runs its channel's
// recursion over the tile's 32 samples, and results leave through the same
// staging with coalesced row stores.  Coefficients live in registers for orders
// up to 16 and in shared memory (one column per lane, conflict-free) above.
#include "common.cuh"
#include "kernels.h"

namespace dfilt {

namespace {

constexpr int kTile = 32;

template <int MB>
struct SeqCoef {
    // REG: coefficients in registers; otherwise per-lane columns in shared memory.
    static constexpr bool REG = MB <= 16;
};

// Per-row metadata of the warp's 32 channels, fetched lane-wise then shuffled.
struct RowInfo {
    int64_t off;
    int len;
};

__device__ __forceinline__ RowInfo row_info(const Channel &c, int r) {
    RowInfo ri;
    ri.off = __shfl_sync(0xffffffffu, c.off, r);
    ri.len = __shfl_sync(0xffffffffu, (int)c.len, r);
    return ri;
}

template <int MB>
__global__ void __launch_bounds__(32) seq_fwd_kernel(const float *__restrict__ x,
                                                     const float *__restrict__ b,
                                                     const float *__restrict__ a,
                                                     const float *__restrict__ zi,
                                                     float *__restrict__ y, Batch bt) {
    constexpr bool REG = SeqCoef<MB>::REG;
    __shared__ float tile[kTile][kTile + 1];
    __shared__ float sa[REG ? 1 : MB][32];
    __shared__ float sb[REG ? 1 : MB + 1][32];

    const int lane = threadIdx.x;
    const int64_t ch = (int64_t)blockIdx.x * 32 + lane;
    const bool valid = ch < bt.B;
    Channel c{0, 0, 1, 0};
    if (valid) c = channel_of(bt, ch);

    float ra[REG ? MB : 1], rb[REG ? MB + 1 : 1], s[MB];
#pragma unroll
    for (int k = 0; k < MB; ++k) {
        float av = (valid && k < c.M) ? a[ch * bt.Mstride + k] : 0.f;
        float zv = (valid && zi && k < c.M) ? zi[ch * bt.Mstride + k] : 0.f;
        s[k] = zv;
        if constexpr (REG) ra[k] = av; else sa[k][lane] = av;
    }
#pragma unroll
    for (int k = 0; k <= MB; ++k) {
        float bv = (valid && k <= c.N) ? b[ch * bt.Nstride + k] : 0.f;
        if constexpr (REG) rb[k] = bv; else sb[k][lane] = bv;
    }
    __syncwarp();

    int tmax = valid ? (int)c.len : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));

    // prefetch the first tile into registers: row r, column lane
    float pre[kTile];
#pragma unroll
    for (int r = 0; r < kTile; ++r) {
        RowInfo ri = row_info(c, r);
        pre[r] = (lane < ri.len) ? x[ri.off + lane] : 0.f;
    }
    for (int t0 = 0; t0 < tmax; t0 += kTile) {
#pragma unroll
        for (int r = 0; r < kTile; ++r) tile[r][lane] = pre[r];
        __syncwarp();
        if (t0 + kTile < tmax) {
#pragma unroll
            for (int r = 0; r < kTile; ++r) {
                RowInfo ri = row_info(c, r);
                int t = t0 + kTile + lane;
                pre[r] = (t < ri.len) ? x[ri.off + t] : 0.f;
            }
        }
        const int nsteps = min(kTile, (int)c.len - t0);   // may be <= 0 for short rows
#pragma unroll 4
        for (int tt = 0; tt < kTile; ++tt) {
            if (tt < nsteps) {
                const float xn = tile[lane][tt];
                const float b0 = REG ? rb[0] : sb[0][lane];
                const float yn = fmaf(b0, xn, s[0]);
#pragma unroll
                for (int k = 0; k < MB; ++k) {
                    const float nxt = (k + 1 < MB) ? s[k + 1] : 0.f;
                    const float bk = REG ? rb[k + 1] : sb[k + 1][lane];
                    const float ak = REG ? ra[k] : sa[k][lane];
                    s[k] = fmaf(-ak, yn, fmaf(bk, xn, nxt));
                }
                tile[lane][tt] = yn;
            }
        }
        __syncwarp();
#pragma unroll 4
        for (int r = 0; r < kTile; ++r) {
            RowInfo ri = row_info(c, r);
            int t = t0 + lane;
            if (t < ri.len) y[ri.off + t] = tile[r][lane];
        }
        __syncwarp();
    }
}

template <int MB>
__global__ void __launch_bounds__(32) seq_bwd_kernel(const float *__restrict__ gy,
                                                     const float *__restrict__ x,
                                                     const float *__restrict__ y,
                                                     const float *__restrict__ b,
                                                     const float *__restrict__ a,
                                                     float *__restrict__ gx, float *__restrict__ gb,
                                                     float *__restrict__ ga,
                                                     float *__restrict__ gzi, Batch bt) {
    constexpr bool REG = SeqCoef<MB>::REG;
    __shared__ float tg[kTile][kTile + 1];
    __shared__ float tx[kTile][kTile + 1];
    __shared__ float ty[kTile][kTile + 1];
    __shared__ float sa[REG ? 1 : MB][32];
    __shared__ float sb[REG ? 1 : MB + 1][32];
    __shared__ float tot[REG ? 1 : 2 * MB + 1][32];   // running totals above order 16

    const int lane = threadIdx.x;
    const int64_t ch = (int64_t)blockIdx.x * 32 + lane;
    const bool valid = ch < bt.B;
    Channel c{0, 0, 1, 0};
    if (valid) c = channel_of(bt, ch);

    float ra[REG ? MB : 1], rb[REG ? MB + 1 : 1];
#pragma unroll
    for (int k = 0; k < MB; ++k) {
        float av = (valid && k < c.M) ? a[ch * bt.Mstride + k] : 0.f;
        if constexpr (REG) ra[k] = av; else sa[k][lane] = av;
    }
#pragma unroll
    for (int k = 0; k <= MB; ++k) {
        float bv = (valid && k <= c.N) ? b[ch * bt.Nstride + k] : 0.f;
        if constexpr (REG) rb[k] = bv; else sb[k][lane] = bv;
    }
    // uh[j] = u[n+1+j] (the next MB adjoint values; zero past the end, App. A)
    float uh[MB];
    // per-tile partial correlations: pb[k] = sum u[n+k] x[n], pa[k] = sum u[n+1+k] y[n]
    float pb[MB + 1], pa[MB];
    float totb[REG ? MB + 1 : 1], tota[REG ? MB : 1];
#pragma unroll
    for (int k = 0; k < MB; ++k) uh[k] = 0.f;
#pragma unroll
    for (int k = 0; k <= MB; ++k) {
        if constexpr (REG) totb[k] = 0.f; else tot[k][lane] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < MB; ++k) {
        if constexpr (REG) tota[k] = 0.f; else tot[MB + 1 + k][lane] = 0.f;
    }
    __syncwarp();

    int tmax = valid ? (int)c.len : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    const int ntiles = (tmax + kTile - 1) / kTile;

    for (int it = ntiles - 1; it >= 0; --it) {
        const int t0 = it * kTile;
#pragma unroll 4
        for (int r = 0; r < kTile; ++r) {
            RowInfo ri = row_info(c, r);
            int t = t0 + lane;
            bool in = t < ri.len;
            tg[r][lane] = in ? gy[ri.off + t] : 0.f;
            tx[r][lane] = in ? x[ri.off + t] : 0.f;
            ty[r][lane] = in ? y[ri.off + t] : 0.f;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k <= MB; ++k) pb[k] = 0.f;
#pragma unroll
        for (int k = 0; k < MB; ++k) pa[k] = 0.f;
        const int nsteps = min(kTile, (int)c.len - t0);
#pragma unroll 2
        for (int tt = kTile - 1; tt >= 0; --tt) {
            if (tt < nsteps) {
                const float gn = tg[lane][tt], xn = tx[lane][tt], yn = ty[lane][tt];
                float un = gn;
#pragma unroll
                for (int k = 0; k < MB; ++k) un = fmaf(-(REG ? ra[k] : sa[k][lane]), uh[k], un);
                float gxn = (REG ? rb[0] : sb[0][lane]) * un;
#pragma unroll
                for (int k = 0; k < MB; ++k) gxn = fmaf(REG ? rb[k + 1] : sb[k + 1][lane], uh[k], gxn);
                pb[0] = fmaf(un, xn, pb[0]);
#pragma unroll
                for (int k = 0; k < MB; ++k) {
                    pb[k + 1] = fmaf(uh[k], xn, pb[k + 1]);
                    pa[k] = fmaf(uh[k], yn, pa[k]);
                }
#pragma unroll
                for (int k = MB - 1; k > 0; --k) uh[k] = uh[k - 1];
                uh[0] = un;
                tg[lane][tt] = gxn;
            }
        }
#pragma unroll
        for (int k = 0; k <= MB; ++k) {
            if constexpr (REG) totb[k] += pb[k]; else tot[k][lane] += pb[k];
        }
#pragma unroll
        for (int k = 0; k < MB; ++k) {
            if constexpr (REG) tota[k] += pa[k]; else tot[MB + 1 + k][lane] += pa[k];
        }
        __syncwarp();
        if (gx) {
#pragma unroll 4
            for (int r = 0; r < kTile; ++r) {
                RowInfo ri = row_info(c, r);
                int t = t0 + lane;
                if (t < ri.len) gx[ri.off + t] = tg[r][lane];
            }
        }
        __syncwarp();
    }
    if (!valid) return;
    if (gb) {
#pragma unroll
        for (int k = 0; k <= MB; ++k)
            if (k <= c.N) gb[ch * bt.Nstride + k] = REG ? totb[k] : tot[k][lane];
    }
    if (ga) {
#pragma unroll
        for (int k = 0; k < MB; ++k)
            if (k < c.M) ga[ch * bt.Mstride + k] = -(REG ? tota[k] : tot[MB + 1 + k][lane]);
    }
    if (gzi) {
#pragma unroll
        for (int k = 0; k < MB; ++k)
            if (k < c.M) gzi[ch * bt.Mstride + k] = uh[k];
    }
}

}  // namespace

int seq_bucket(int M) {
    for (int mb : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64})
        if (M <= mb) return mb;
    return -1;
}

#define DFILT_SEQ_CASES(X) X(1) X(2) X(3) X(4) X(6) X(8) X(12) X(16) X(24) X(32) X(48) X(64)

cudaError_t launch_seq_fwd(const float *x, const float *b, const float *a, const float *zi,
                           float *y, const Batch &bt, int Mmax, cudaStream_t st) {
    if (bt.B == 0) return cudaSuccess;
    const int mb = seq_bucket(Mmax);
    const dim3 grid((unsigned)((bt.B + 31) / 32)), block(32);
    switch (mb) {
#define X(MB) \
    case MB: seq_fwd_kernel<MB><<<grid, block, 0, st>>>(x, b, a, zi, y, bt); note_launch(); break;
        DFILT_SEQ_CASES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_seq_bwd(const float *gy, const float *x, const float *y, const float *b,
                           const float *a, float *gx, float *gb, float *ga, float *gzi,
                           const Batch &bt, int Mmax, cudaStream_t st) {
    if (bt.B == 0) return cudaSuccess;
    const int mb = seq_bucket(Mmax);
    const dim3 grid((unsigned)((bt.B + 31) / 32)), block(32);
    switch (mb) {
#define X(MB)                                                                               \
    case MB:                                                                                \
        seq_bwd_kernel<MB><<<grid, block, 0, st>>>(gy, x, y, b, a, gx, gb, ga, gzi, bt); note_launch();    \
        break;
        DFILT_SEQ_CASES(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dfilt
