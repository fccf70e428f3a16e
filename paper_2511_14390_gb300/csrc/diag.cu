// The App. B recurrence with A diagonalised (the paper's Diag-EXT, Sec. 3.2 and Sec. 4):
// A = V diag(lam) V^-1 with complex lam, V, V^-1 per channel.  In the eigenbasis
// q = V^-1 v the recurrence is element by element,
//     q(n+1) = lam * q(n) + V^-1 z(n),   q(0) = V^-1 v0,   v(n) = Re(V q(n)),
// so combining two steps costs M complex multiply-adds instead of an M x M product; the
// projections V^-1 z and V q (the "eigen-space projection" Sec. 4 names) are fused into
// the scan's passes.  Backward (App. A, Eqs. dLdz and dLdvBA): dL/dz is the same operator
// for A^T = V^-T diag(lam) V^T (the transposed pair) on the time-reversed dL/dv from a
// zero state; dL/dv(0) = A^T dL/dz(0); dL/dA = sum_n dL/dz(n) v(n)^T with v(n) the state
// before step n.
//
// Chunked scan on the CUDA cores (M <= 4: a few complex FMAs per step, HBM-bound):
//   * a warp owns a segment of 1024 steps, staged in shared memory with coalesced
//     float4 loads; lane j runs the recurrence over its 32-step chunk from a zero state
//     (chunk end e_j), and a warp shuffle scan with lam^(32 * 2^k) turns the e_j into
//     the chunks' entry states;
//   * pass 1 keeps only the segment's aggregate; a carry kernel (one thread per channel
//     and mode) steps the segment entries q_{g+1} = lam^1024 q_g + agg_g;
//   * pass 2 reruns each chunk from its true entry in shared memory, v = Re(V q)
//     replacing z, and stores v with float4 stores.
// Complex FP32: in the eigenbasis the transition is diagonal with |lam| < 1, so rounding
// errors are not amplified by transient growth; the powers lam^(2^k) come from FP64
// squaring.  z is read twice and v written once; dL/dA sums over 1024 steps in FP32 and
// across segments in FP64, in a fixed order.
#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

using namespace dfilt;

namespace {

constexpr int kDgChunk = 32;                    // steps per lane
constexpr int kDgSeg = 32 * kDgChunk;           // steps per warp (segment)
constexpr int kDgWarps = 4;                     // segments per block
constexpr int kDgPow = 6;                       // lam^(32 * 2^k), k = 0..5 (5: lam^1024)
constexpr int kDgMaxM = 4;

size_t al256(size_t n) { return (n + 255) / 256 * 256; }

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {   // a * b + c
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return cfma(a, b, make_float2(0.f, 0.f)); }

struct DgArgs {
    const float2 *lam;   // [B][M]
    const float2 *V;     // [B][M][M] row-major
    const float2 *Vinv;  // [B][M][M]
    int trans;           // 0: the pair (V, V^-1) of A; 1: the pair (V^-T, V^T) of A^T
    const float2 *pw;    // [B][kDgPow][M]
    const float *z;      // [B][T][M] input of the pass
    float *out;          // [B][T][M] output of the pass
    const float2 *seg_in;   // [B][G][M] segment entry states (pass 2)
    float2 *agg;            // [B][G][M] segment aggregates (pass 1)
    int64_t B, T, G, groups;
};

// lam^(32 * 2^k), k = 0..5, per channel and mode, by FP64 squaring.
template <int M>
__global__ void dg_setup_kernel(const float2 *__restrict__ lam, float2 *__restrict__ pw, int64_t B) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * M) return;
    const int64_t b = i / M;
    const int m = (int)(i - b * M);
    double re = lam[i].x, im = lam[i].y;
    for (int k = 1; k <= 10; ++k) {   // lam^(2^k)
        const double r2 = re * re - im * im, i2 = 2.0 * re * im;
        re = r2;
        im = i2;
        if (k >= 5) pw[(b * kDgPow + (k - 5)) * M + m] = make_float2((float)re, (float)im);
    }
}

// One pass over the segments (FINAL = false: segment aggregates; true: outputs).  REV runs
// logical step i at memory position T-1-i.  Block = kDgWarps segments of one channel.
template <int M, bool REV, bool FINAL>
__global__ void __launch_bounds__(32 * kDgWarps) dg_seg_kernel(DgArgs d) {
    constexpr int ROW = kDgChunk * M + 1;           // padded chunk row (conflict-free lanes)
    extern __shared__ float smem[];
    float *zs = smem + (threadIdx.x >> 5) * (32 * ROW);
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x / d.groups;
    const int64_t g = ((int64_t)blockIdx.x - b * d.groups) * kDgWarps + (threadIdx.x >> 5);
    if (g >= d.G) return;                           // whole warp leaves together

    float2 lam[M], P[M][M], Q[M][M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        lam[i] = d.lam[b * M + i];
#pragma unroll
        for (int j = 0; j < M; ++j) {
            // input projection P (V^-1, or V^T) and output projection Q (V, or V^-T)
            P[i][j] = d.trans ? d.V[(b * M + j) * M + i] : d.Vinv[(b * M + i) * M + j];
            Q[i][j] = d.trans ? d.Vinv[(b * M + j) * M + i] : d.V[(b * M + i) * M + j];
        }
    }

    const int cnt = (int)((d.T - g * kDgSeg) < kDgSeg ? (d.T - g * kDgSeg) : kDgSeg);
    const int64_t p0 = REV ? d.T - g * kDgSeg - cnt : g * kDgSeg;   // memory positions [p0, p0+cnt)
    const float *zb = d.z + (b * d.T + p0) * M;
    auto slot = [&](int f) {                        // shared-memory slot of segment float f
        const int pr = f / M, m = f - pr * M;
        const int l = REV ? cnt - 1 - pr : pr;
        return (l >> 5) * ROW + (l & 31) * M + m;
    };
    // every segment starts on a 16-byte boundary when T*M is a multiple of 4
    const bool vec = ((d.T * M) & 3) == 0 && (reinterpret_cast<uintptr_t>(d.z) & 15) == 0 &&
                     (!FINAL || (reinterpret_cast<uintptr_t>(d.out) & 15) == 0);
    const int nf = cnt * M;
    int done = 0;
    if (vec) {
        constexpr int R = 8;                        // float4 loads in flight per lane
        const float4 *z4 = reinterpret_cast<const float4 *>(zb);
        const int n4 = nf >> 2;
        for (int q0 = 0; q0 < n4; q0 += 32 * R) {
            float4 r4[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int q = q0 + r * 32 + lane;
                r4[r] = q < n4 ? __ldg(z4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
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
    for (int f = done + lane; f < nf; f += 32) zs[slot(f)] = __ldg(zb + f);
    __syncwarp();

    // this lane's chunk: logical steps [32 lane, 32 lane + n) of the segment
    const int n = cnt - 32 * lane < 0 ? 0 : (cnt - 32 * lane > kDgChunk ? kDgChunk : cnt - 32 * lane);
    float *row = zs + lane * ROW;
    float2 q[M];
#pragma unroll
    for (int m = 0; m < M; ++m) q[m] = make_float2(0.f, 0.f);
    auto step = [&](int s, float2 (&st)[M]) {       // st <- lam st + P z(s)
        float zz[M];
#pragma unroll
        for (int m = 0; m < M; ++m) zz[m] = row[s * M + m];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            float2 w = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < M; ++j) w = make_float2(fmaf(P[i][j].x, zz[j], w.x), fmaf(P[i][j].y, zz[j], w.y));
            st[i] = cfma(lam[i], st[i], w);
        }
    };
#pragma unroll 4
    for (int s = 0; s < n; ++s) step(s, q);

    // inclusive warp scan of the chunk ends with the chunk transition lam^32
    float2 inc[M];
#pragma unroll
    for (int m = 0; m < M; ++m) inc[m] = q[m];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int dd = 1 << k;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const float2 pk = d.pw[(b * kDgPow + k) * M + m];
            float2 o;
            o.x = __shfl_up_sync(0xffffffffu, inc[m].x, dd);
            o.y = __shfl_up_sync(0xffffffffu, inc[m].y, dd);
            if (lane >= dd) inc[m] = cfma(pk, o, inc[m]);
        }
    }
    if constexpr (!FINAL) {
        if (lane == 31) {
#pragma unroll
            for (int m = 0; m < M; ++m) d.agg[(b * d.G + g) * M + m] = inc[m];
        }
        return;
    } else {
        // the chunk's entry: the lanes before it, then the segment entry carried over
        // lane * 32 steps (lam^(32 lane) from the bits of the lane index)
#pragma unroll
        for (int m = 0; m < M; ++m) {
            float2 ex;
            ex.x = __shfl_up_sync(0xffffffffu, inc[m].x, 1);
            ex.y = __shfl_up_sync(0xffffffffu, inc[m].y, 1);
            if (lane == 0) ex = make_float2(0.f, 0.f);
            float2 pl = make_float2(1.f, 0.f);
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if ((lane >> k) & 1) pl = cmul(pl, d.pw[(b * kDgPow + k) * M + m]);
            q[m] = cfma(pl, d.seg_in[(b * d.G + g) * M + m], ex);
        }
        // rerun the chunk from its entry; v = Re(Q q) replaces z in shared memory
#pragma unroll 4
        for (int s = 0; s < n; ++s) {
            step(s, q);
#pragma unroll
            for (int i = 0; i < M; ++i) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < M; ++j) acc = fmaf(Q[i][j].x, q[j].x, fmaf(-Q[i][j].y, q[j].y, acc));
                row[s * M + i] = acc;
            }
        }
        __syncwarp();
        float *ob = d.out + (b * d.T + p0) * M;
        int odone = 0;
        if (vec) {
            float4 *o4 = reinterpret_cast<float4 *>(ob);
            const int n4 = nf >> 2;
            for (int qq = lane; qq < n4; qq += 32)
                o4[qq] = make_float4(zs[slot(4 * qq)], zs[slot(4 * qq + 1)], zs[slot(4 * qq + 2)],
                                     zs[slot(4 * qq + 3)]);
            odone = n4 * 4;
        }
        for (int f = odone + lane; f < nf; f += 32) ob[f] = zs[slot(f)];
    }
}

// Segment entry states: q_0 = P v0 (forward) or 0, q_{g+1} = lam^1024 q_g + agg_g.
template <int M>
__global__ void dg_carry_kernel(DgArgs d, const float *__restrict__ v0, float2 *__restrict__ seg_in) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.B * M) return;
    const int64_t b = i / M;
    const int m = (int)(i - b * M);
    float2 q = make_float2(0.f, 0.f);
    if (v0) {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const float2 p = d.trans ? d.V[(b * M + j) * M + m] : d.Vinv[(b * M + m) * M + j];
            q.x = fmaf(p.x, v0[b * M + j], q.x);
            q.y = fmaf(p.y, v0[b * M + j], q.y);
        }
    }
    const float2 L = d.pw[(b * kDgPow + 5) * M + m];
    for (int64_t g = 0; g < d.G; ++g) {
        seg_in[(b * d.G + g) * M + m] = q;
        q = cfma(L, q, d.agg[(b * d.G + g) * M + m]);
    }
}

// dL/dA partial sums per 1024-step segment: sum_n gz(n) v(n)^T, v(n) the state before
// step n (v0 for n = 0); FP32 per thread over 4 steps, a fixed-order tree over the
// block, stored as FP64.
template <int M>
__global__ void __launch_bounds__(256) dg_grada_kernel(const float *__restrict__ gz,
                                                       const float *__restrict__ v,
                                                       const float *__restrict__ v0,
                                                       double *__restrict__ part, int64_t T,
                                                       int64_t G) {
    __shared__ float red[8][M * M];
    const int64_t b = blockIdx.x / G, g = blockIdx.x - b * G;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float acc[M * M];
#pragma unroll
    for (int e = 0; e < M * M; ++e) acc[e] = 0.f;
    for (int s = 0; s < kDgSeg / 256; ++s) {
        const int64_t nstep = g * kDgSeg + t * (kDgSeg / 256) + s;
        if (nstep >= T) break;
        const float *gp = gz + (b * T + nstep) * M;
        const float *vp = nstep == 0 ? (v0 ? v0 + b * M : nullptr) : v + (b * T + nstep - 1) * M;
        if (!vp) continue;
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = 0; j < M; ++j) acc[i * M + j] = fmaf(gp[i], vp[j], acc[i * M + j]);
    }
#pragma unroll
    for (int e = 0; e < M * M; ++e) {
        float x = acc[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][e] = x;
    }
    __syncthreads();
    if (t < M * M) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += (double)red[w][t];
        part[(b * G + g) * M * M + t] = s;
    }
}

// dL/dA = sum over segments in order (FP64); dL/dv(0) = Re(V^-T (lam * (V^T gz(0)))).
template <int M>
__global__ void dg_grada_final_kernel(const double *__restrict__ part, const float2 *__restrict__ lam,
                                      const float2 *__restrict__ V, const float2 *__restrict__ Vinv,
                                      const float *__restrict__ gz, float *__restrict__ gA,
                                      float *__restrict__ gv0, int64_t B, int64_t T, int64_t G) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * M * M) return;
    const int64_t b = i / (M * M);
    const int e = (int)(i - b * M * M);
    if (gA) {
        double s = 0.0;
        for (int64_t g = 0; g < G; ++g) s += part[(b * G + g) * M * M + e];
        gA[b * M * M + e] = (float)s;
    }
    if (gv0 && e < M) {
        if (T == 0) {
            gv0[b * M + e] = 0.f;
            return;
        }
        const float *g0 = gz + b * T * M;
        // u = lam * (V^T gz(0)); dL/dv0[e] = Re(sum_m Vinv[m][e] u[m])
        double re = 0.0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            double ur = 0.0, ui = 0.0;
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const float2 vv = V[(b * M + j) * M + m];
                ur += (double)vv.x * g0[j];
                ui += (double)vv.y * g0[j];
            }
            const float2 l = lam[b * M + m];
            const double wr = l.x * ur - l.y * ui, wi = l.x * ui + l.y * ur;
            const float2 vi = Vinv[(b * M + m) * M + e];
            re += (double)vi.x * wr - (double)vi.y * wi;
        }
        gv0[b * M + e] = (float)re;
    }
}

struct DgLayout {
    int64_t G;
    size_t pw, agg, seg, part, fwd_total, bwd_total;
};

DgLayout dg_layout(int64_t B, int64_t T, int M) {
    DgLayout L{};
    L.G = (T + kDgSeg - 1) / kDgSeg;
    size_t o = 0;
    L.pw = o;
    o += al256((size_t)B * kDgPow * M * 8);
    L.agg = o;
    o += al256((size_t)B * L.G * M * 8);
    L.seg = o;
    o += al256((size_t)B * L.G * M * 8);
    L.fwd_total = o;
    L.part = o;
    o += al256((size_t)B * L.G * M * M * 8);
    L.bwd_total = o;
    return L;
}

template <int M, bool REV>
cudaError_t dg_scan(DgArgs d, const float *v0, char *ws, const DgLayout &L, cudaStream_t st) {
    float2 *pw = reinterpret_cast<float2 *>(ws + L.pw);
    d.pw = pw;
    d.agg = reinterpret_cast<float2 *>(ws + L.agg);
    float2 *seg_in = reinterpret_cast<float2 *>(ws + L.seg);
    d.seg_in = seg_in;
    d.G = L.G;
    const int64_t nbm = d.B * M;
    dg_setup_kernel<M><<<(unsigned)((nbm + 127) / 128), 128, 0, st>>>(d.lam, pw, d.B); note_launch();
    if (L.G == 0) return cudaGetLastError();
    d.groups = (L.G + kDgWarps - 1) / kDgWarps;
    const int64_t blocks = d.B * d.groups;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)kDgWarps * 32 * (kDgChunk * M + 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(dg_seg_kernel<M, REV, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(dg_seg_kernel<M, REV, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dg_seg_kernel<M, REV, false><<<(unsigned)blocks, 32 * kDgWarps, smem, st>>>(d); note_launch();
    dg_carry_kernel<M><<<(unsigned)((nbm + 127) / 128), 128, 0, st>>>(d, v0, seg_in); note_launch();
    dg_seg_kernel<M, REV, true><<<(unsigned)blocks, 32 * kDgWarps, smem, st>>>(d); note_launch();
    return cudaGetLastError();
}

template <int M>
cudaError_t dg_forward_m(const float2 *lam, const float2 *V, const float2 *Vinv, const float *v0,
                         const float *z, float *v, char *ws, const DgLayout &L, int64_t B,
                         int64_t T, cudaStream_t st) {
    DgArgs d{};
    d.lam = lam;
    d.V = V;
    d.Vinv = Vinv;
    d.trans = 0;
    d.z = z;
    d.out = v;
    d.B = B;
    d.T = T;
    return dg_scan<M, false>(d, v0, ws, L, st);
}

template <int M>
cudaError_t dg_backward_m(const float2 *lam, const float2 *V, const float2 *Vinv, const float *v0,
                          const float *v, const float *gv, float *gA, float *gv0, float *gz,
                          char *ws, const DgLayout &L, int64_t B, int64_t T, cudaStream_t st) {
    DgArgs d{};
    d.lam = lam;
    d.V = V;
    d.Vinv = Vinv;
    d.trans = 1;
    d.z = gv;
    d.out = gz;
    d.B = B;
    d.T = T;
    cudaError_t e = dg_scan<M, true>(d, nullptr, ws, L, st);
    if (e != cudaSuccess) return e;
    double *part = reinterpret_cast<double *>(ws + L.part);
    if (gA && L.G > 0) {
        const int64_t blocks = B * L.G;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        dg_grada_kernel<M><<<(unsigned)blocks, 256, 0, st>>>(gz, v, v0, part, T, L.G); note_launch();
    }
    if (gA || gv0) {
        const int64_t n = B * M * M;
        dg_grada_final_kernel<M><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, lam, V, Vinv, gz,
                                                                           gA, gv0, B, T, L.G); note_launch();
    }
    return cudaGetLastError();
}

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

dfilt_status to_status(cudaError_t e) { return e == cudaSuccess ? DFILT_OK : DFILT_ERR_CUDA; }

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

}  // namespace

extern "C" dfilt_status dfilt_diag_workspace_size(int64_t B, int64_t T, int M, size_t *fwd_ws,
                                                  size_t *bwd_ws) {
    if (B < 0 || T < 0 || M < 1) return DFILT_ERR_INVALID_ARG;
    if (M > kDgMaxM) return DFILT_ERR_UNSUPPORTED;
    const DgLayout L = dg_layout(B, T, M);
    if (fwd_ws) *fwd_ws = L.fwd_total;
    if (bwd_ws) *bwd_ws = L.bwd_total;
    return DFILT_OK;
}

extern "C" dfilt_status dfilt_diag_forward(const float *lam, const float *V, const float *Vinv,
                                           const float *v0, const float *z, float *v, void *ws,
                                           size_t ws_bytes, int64_t B, int64_t T, int M,
                                           void *stream) {
    NvtxRange range("dfilt_diag_forward");
    if (B < 0 || T < 0 || M < 1) return DFILT_ERR_INVALID_ARG;
    if (M > kDgMaxM) return DFILT_ERR_UNSUPPORTED;
    if (B == 0 || T == 0) return DFILT_OK;
    if (!lam || !V || !Vinv || !z || !v) return DFILT_ERR_INVALID_ARG;
    if (!aligned8(lam) || !aligned8(V) || !aligned8(Vinv)) return DFILT_ERR_INVALID_ARG;
    const DgLayout L = dg_layout(B, T, M);
    if (!ws || ws_bytes < L.fwd_total) return DFILT_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & 15) return DFILT_ERR_INVALID_ARG;
    char *w = static_cast<char *>(ws);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float2 *l2 = reinterpret_cast<const float2 *>(lam);
    const float2 *V2 = reinterpret_cast<const float2 *>(V);
    const float2 *Vi2 = reinterpret_cast<const float2 *>(Vinv);
    switch (M) {
        case 1: return to_status(dg_forward_m<1>(l2, V2, Vi2, v0, z, v, w, L, B, T, st));
        case 2: return to_status(dg_forward_m<2>(l2, V2, Vi2, v0, z, v, w, L, B, T, st));
        case 3: return to_status(dg_forward_m<3>(l2, V2, Vi2, v0, z, v, w, L, B, T, st));
        default: return to_status(dg_forward_m<4>(l2, V2, Vi2, v0, z, v, w, L, B, T, st));
    }
}

extern "C" dfilt_status dfilt_diag_backward(const float *lam, const float *V, const float *Vinv,
                                            const float *v0, const float *v, const float *gv,
                                            float *gA, float *gv0, float *gz, void *ws,
                                            size_t ws_bytes, int64_t B, int64_t T, int M,
                                            void *stream) {
    NvtxRange range("dfilt_diag_backward");
    if (B < 0 || T < 0 || M < 1) return DFILT_ERR_INVALID_ARG;
    if (M > kDgMaxM) return DFILT_ERR_UNSUPPORTED;
    if (B == 0) return DFILT_OK;
    if (!lam || !V || !Vinv || !gz || (T > 0 && !gv) || (gA && T > 0 && !v)) return DFILT_ERR_INVALID_ARG;
    if (!aligned8(lam) || !aligned8(V) || !aligned8(Vinv)) return DFILT_ERR_INVALID_ARG;
    const DgLayout L = dg_layout(B, T, M);
    if (!ws || ws_bytes < L.bwd_total) return DFILT_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & 15) return DFILT_ERR_INVALID_ARG;
    char *w = static_cast<char *>(ws);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float2 *l2 = reinterpret_cast<const float2 *>(lam);
    const float2 *V2 = reinterpret_cast<const float2 *>(V);
    const float2 *Vi2 = reinterpret_cast<const float2 *>(Vinv);
    switch (M) {
        case 1: return to_status(dg_backward_m<1>(l2, V2, Vi2, v0, v, gv, gA, gv0, gz, w, L, B, T, st));
        case 2: return to_status(dg_backward_m<2>(l2, V2, Vi2, v0, v, gv, gA, gv0, gz, w, L, B, T, st));
        case 3: return to_status(dg_backward_m<3>(l2, V2, Vi2, v0, v, gv, gA, gv0, gz, w, L, B, T, st));
        default: return to_status(dg_backward_m<4>(l2, V2, Vi2, v0, v, gv, gA, gv0, gz, w, L, B, T, st));
    }
}
