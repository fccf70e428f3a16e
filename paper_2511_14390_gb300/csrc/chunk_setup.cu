// Coefficient setup of the chunked algorithm: per channel, the impulse responses, the
// free-response and end-state blocks, and the chunk transition of the chunk algebra
// (see chunk.cuh), formed in extended precision and rounded to the operand precision.
// One launch writes the forward records, the backward records, or both.
//
// GB300's FP64 pipe is narrow and a warp-wide FP64 instruction costs it the same
// whether 1 or 32 lanes are active, so both variants keep every lane busy:
//   * low orders (MB <= 4): one warp per channel in double-word arithmetic
//     (dword.cuh) on the full-rate FP32 pipes; one serial recurrence for the
//     all-pole impulse response, then every table entry as a short sum over it;
//   * higher orders with the double-word scan (the automatic choice above order 2):
//     one block per channel, the same closed forms in FP64, the impulse response's
//     recurrence shared by a warp and every entry summed in parallel (setup_hi_kernel,
//     below);
//   * higher orders with the forced FP32 scan (FP32 powers of the transition): FP64, one
//     block per channel, thread m evolves column m of F^i (i = 0..L) and every table is
//     read off those columns in parallel:
//       O_L[i][m] = (F^i e_m)[0],  g[n] = sum_m Gv_m O_L[n-1][m] (n >= 1),
//       h[n] likewise with the all-pole input vector, R_L[:, L-1-i] = F^i Gv
//       (a reduction over the columns held in shared memory), Abar = F^L
//     (L successive companion products: companion-matrix powers of high-order
//     filters grow transiently by orders of magnitude, and repeated squaring loses
//     accuracy on them).  The backward's O^u columns run the anti-causal all-pole
//     recursion from a unit future state, one column per thread.
#include "chunk.cuh"
#include "chunk_pipe.cuh"
#include "dword.cuh"

namespace dfilt {

namespace {

// ---------------------------------------------------------------------------
// low orders: one warp per channel, double-word arithmetic on the FP32 pipes.
// Every table is a short sum over the all-pole impulse response h (the impulse
// response of 1/A) and the coefficients, so after one serial recurrence for h
// (lane 0) the lanes fill the tables in parallel, with coalesced stores.  With the
// TDF-II state s_k[n] = sum_{j>k} (b_j x[n+k-j] - a_j y[n+k-j]) (n >= M):
//   g[n]        = sum_k b_k h[n-k]                       (impulse response of B/A)
//   O_L[i][m]   = h[i-m]                                 (zi enters as an injected input)
//   R_L[k][j]   = b_t - sum_{l>k} a_l g[t-l],   t = L+k-j
//   Abar[k][m]  = -sum_{l>k} a_l h[L+k-l-m]
//   O^u[n][m]   = -sum_{j<=min(L-1-n, MB-1-m)} a_{j+1+m} h[L-1-n-j]
//                 (the adjoint recursion in reversed time, its future values turned
//                  into injected inputs)
//   O^gx[n][m]  = sum_k b_k U(n+k, m),  U(p, m) = O^u[p][m] (p < L), [p-L == m] else
//   Abar'[k][m] = O^u[k][m]
// ---------------------------------------------------------------------------
constexpr int kSmallWarps = 4;   // channels per block

template <int MB>
struct SmallScratch {
    float hhi[kL + MB], hlo[kL + MB];   // h[0 .. L+MB)
    float ghi[kL], glo[kL];             // g[0 .. L)
    float uhi[kL * MB], ulo[kL * MB];   // O^u (backward)
    float ahi[2][MB * MB], alo[2][MB * MB];
};

template <int MB>
__global__ void __launch_bounds__(32 * kSmallWarps) setup_small_kernel(
    const float *__restrict__ b, const float *__restrict__ a, char *__restrict__ fwd_tabs,
    char *__restrict__ bwd_tabs, unsigned long long *__restrict__ counter, Batch bt, bool f64) {
    using Tab = ChunkTab<MB>;
    constexpr int L = kL;
    __shared__ SmallScratch<MB> scr_all[kSmallWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    SmallScratch<MB> &sc = scr_all[wib];
    if (counter && blockIdx.x == 0 && threadIdx.x == 0) *counter = 0ull;
    int64_t ch;
    if (!work_channel(bt, (int64_t)blockIdx.x * kSmallWarps + wib, &ch)) return;
    const Channel c = channel_of(bt, ch);
    dw av[MB], bp[MB + 1];   // av[k] = a_{k+1}; zero past the channel's orders
#pragma unroll
    for (int k = 0; k < MB; ++k) av[k] = dw_make(k < c.M ? a[ch * bt.Mstride + k] : 0.f);
#pragma unroll
    for (int k = 0; k <= MB; ++k) bp[k] = dw_make(k <= c.N ? b[ch * bt.Nstride + k] : 0.f);
    auto H = [&](int n) -> dw { return n >= 0 ? dw{sc.hhi[n], sc.hlo[n]} : dw_make(0.f); };
    auto G = [&](int n) -> dw { return n >= 0 ? dw{sc.ghi[n], sc.glo[n]} : dw_make(0.f); };
    // h by the all-pole difference equation (the one serial chain; the oldest terms
    // first, so that only the newest product and difference lie on the chain)
    if (lane == 0) {
        dw wh[MB];
#pragma unroll
        for (int k = 0; k < MB; ++k) wh[k] = dw_make(0.f);
        for (int n = 0; n < L + MB; ++n) {
            dw yh = dw_make(n == 0 ? 1.f : 0.f);
#pragma unroll
            for (int k = MB - 1; k >= 0; --k) yh = yh - av[k] * wh[k];
#pragma unroll
            for (int k = MB - 1; k > 0; --k) wh[k] = wh[k - 1];
            wh[0] = yh;
            sc.hhi[n] = yh.hi;
            sc.hlo[n] = yh.lo;
        }
    }
    __syncwarp();
    const size_t fstride = bt.fwd_stride ? (size_t)bt.fwd_stride : Tab::fwd_rec(f64);
    const size_t bstride = bt.bwd_stride ? (size_t)bt.bwd_stride : Tab::bwd_rec(f64);
    char *RF = fwd_tabs ? fwd_tabs + (size_t)ch * fstride : nullptr;
    char *RB = bwd_tabs ? bwd_tabs + (size_t)ch * bstride : nullptr;
    for (int n = lane; n < L; n += 32) {
        dw acc = dw_make(0.f);
#pragma unroll
        for (int k = 0; k <= MB; ++k) acc = acc + bp[k] * H(n - k);
        sc.ghi[n] = acc.hi;
        sc.glo[n] = acc.lo;
        const float gv = dw_to_float(acc);
        if (RF) reinterpret_cast<float *>(RF + Tab::F_G)[n] = gv;
        if (RB) reinterpret_cast<float *>(RB + Tab::B_G)[n] = gv;
    }
    __syncwarp();
    // the scan block of a record from the transition in sc.a[0]
    auto write_scan = [&](char *S) {
        if (f64) {   // the serial scan's transition: double words (hi, lo), column-major
            float2 *At = reinterpret_cast<float2 *>(S);
            if (lane < MB * MB) {
                const int j = lane / MB, m = lane % MB;   // At[j][m] = A[m][j]
                At[lane] = make_float2(sc.ahi[0][m * MB + j], sc.alo[0][m * MB + j]);
            }
            if constexpr (Tab::kBlockScan) {   // then A^4, by squaring twice
                __syncwarp();
                int cur = 0;
                for (int sq = 0; sq < 2; ++sq) {
                    if (lane < MB * MB) {
                        const int i = lane / MB, j = lane % MB;
                        dw acc = dw_make(0.f);
#pragma unroll
                        for (int k = 0; k < MB; ++k)
                            acc = acc + dw{sc.ahi[cur][i * MB + k], sc.alo[cur][i * MB + k]} *
                                            dw{sc.ahi[cur][k * MB + j], sc.alo[cur][k * MB + j]};
                        sc.ahi[cur ^ 1][lane] = acc.hi;
                        sc.alo[cur ^ 1][lane] = acc.lo;
                    }
                    __syncwarp();
                    cur ^= 1;
                }
                if (lane < MB * MB) {
                    const int j = lane / MB, m = lane % MB;
                    At[MB * MB + lane] = make_float2(sc.ahi[cur][m * MB + j], sc.alo[cur][m * MB + j]);
                }
            }
        } else {
            float *P = reinterpret_cast<float *>(S);
            int cur = 0;
            for (int kp = 0; kp < Tab::NPOW; ++kp) {
                if (lane < MB * MB) P[kp * MB * MB + lane] = dw_to_float(dw{sc.ahi[cur][lane], sc.alo[cur][lane]});
                if (kp + 1 == Tab::NPOW) break;
                if (lane < MB * MB) {
                    const int i = lane / MB, j = lane % MB;
                    dw acc = dw_make(0.f);
#pragma unroll
                    for (int k = 0; k < MB; ++k)
                        acc = acc + dw{sc.ahi[cur][i * MB + k], sc.alo[cur][i * MB + k]} *
                                        dw{sc.ahi[cur][k * MB + j], sc.alo[cur][k * MB + j]};
                    sc.ahi[cur ^ 1][lane] = acc.hi;
                    sc.alo[cur ^ 1][lane] = acc.lo;
                }
                __syncwarp();
                cur ^= 1;
            }
        }
        __syncwarp();
    };
    if (RF) {
        float *RL = reinterpret_cast<float *>(RF + Tab::F_RL);
        float *OL = reinterpret_cast<float *>(RF + Tab::F_OL);
        for (int idx = lane; idx < L * MB; idx += 32) {
            const int i = idx / MB, m = idx % MB;
            OL[idx] = dw_to_float(H(i - m));
        }
        for (int idx = lane; idx < MB * L; idx += 32) {
            const int k = idx / L, j = idx % L, t = L + k - j;
            dw acc = dw_make(0.f);
#pragma unroll
            for (int l = 1; l <= MB; ++l)
                if (l == t) acc = bp[l];
#pragma unroll
            for (int l = 1; l <= MB; ++l)
                if (l > k) acc = acc - av[l - 1] * G(t - l);
            RL[idx] = dw_to_float(acc);
        }
        if (lane < MB * MB) {
            const int k = lane / MB, m = lane % MB;
            dw acc = dw_make(0.f);
#pragma unroll
            for (int l = 1; l <= MB; ++l)
                if (l > k) acc = acc - av[l - 1] * H(L + k - l - m);
            sc.ahi[0][lane] = acc.hi;
            sc.alo[0][lane] = acc.lo;
        }
        __syncwarp();
        write_scan(RF + Tab::F_SCAN);
    }
    if (RB) {
        float *h = reinterpret_cast<float *>(RB + Tab::B_H);
        float *Ou = reinterpret_cast<float *>(RB + Tab::B_OU);
        float *Ogx = reinterpret_cast<float *>(RB + Tab::B_OGX);
        for (int n = lane; n < L; n += 32) h[n] = dw_to_float(H(n));
        for (int idx = lane; idx < L * MB; idx += 32) {
            const int n = idx / MB, m = idx % MB;
            dw acc = dw_make(0.f);
#pragma unroll
            for (int j = 0; j < MB; ++j)
                if (j <= L - 1 - n && j <= MB - 1 - m) acc = acc - av[j + m] * H(L - 1 - n - j);
            sc.uhi[idx] = acc.hi;
            sc.ulo[idx] = acc.lo;
            Ou[idx] = dw_to_float(acc);
        }
        __syncwarp();
        for (int idx = lane; idx < L * MB; idx += 32) {
            const int n = idx / MB, m = idx % MB;
            dw acc = dw_make(0.f);
#pragma unroll
            for (int k = 0; k <= MB; ++k) {
                const int p = n + k;
                if (p < L) acc = acc + bp[k] * dw{sc.uhi[p * MB + m], sc.ulo[p * MB + m]};
                else if (p - L == m) acc = acc + bp[k];
            }
            Ogx[idx] = dw_to_float(acc);
        }
        float *C = reinterpret_cast<float *>(RB + Tab::b_coef(f64));
        for (int k = lane; k < 2 * MB + 1; k += 32)
            C[k] = k < MB ? (k < c.M ? a[ch * bt.Mstride + k] : 0.f)
                          : (k - MB <= c.N ? b[ch * bt.Nstride + (k - MB)] : 0.f);
        if (lane < MB * MB) {
            sc.ahi[0][lane] = sc.uhi[lane];   // Abar'[k][m] = O^u[k][m], k < MB
            sc.alo[0][lane] = sc.ulo[lane];
        }
        __syncwarp();
        write_scan(RB + Tab::B_SCAN);
    }
}

// ---------------------------------------------------------------------------
// higher orders: one block per channel, column-parallel
// ---------------------------------------------------------------------------
template <int MB>
constexpr size_t setup_large_smem() {
    return (size_t)(4 * MB + 1) * 8 + (size_t)(2 * MB + kL) * (MB + 1) * 8;
}

template <int MB>
__global__ void __launch_bounds__(MB) setup_large_kernel(
    const float *__restrict__ b, const float *__restrict__ a, char *__restrict__ fwd_tabs,
    char *__restrict__ bwd_tabs, unsigned long long *__restrict__ counter, Batch bt, bool f64) {
    using Tab = ChunkTab<MB>;
    constexpr int L = kL;
    extern __shared__ double sdyn[];
    double *sa = sdyn, *sbp = sa + MB, *sG = sbp + MB + 1, *sGh = sG + MB;
    // columns of F^i at the current step (row k, col m), the transition, first rows
    double(*sX)[MB + 1] = reinterpret_cast<double(*)[MB + 1]>(sGh + MB);
    double(*sA)[MB + 1] = sX + MB;
    double(*sOL)[MB + 1] = sA + MB;

    const int m = threadIdx.x;
    if (counter && blockIdx.x == 0 && blockIdx.y == 0 && m == 0) *counter = 0ull;
    // grid.y selects the record: forward tables, backward tables, or both
    const bool backward = fwd_tabs == nullptr || blockIdx.y == 1;
    int64_t ch;
    if (!work_channel(bt, (int64_t)blockIdx.x, &ch)) return;   // uniform across the block
    const Channel c = channel_of(bt, ch);
    sa[m] = m < c.M ? (double)a[ch * bt.Mstride + m] : 0.0;
    sbp[m] = m <= c.N ? (double)b[ch * bt.Nstride + m] : 0.0;
    if (m == 0) sbp[MB] = MB <= c.N ? (double)b[ch * bt.Nstride + MB] : 0.0;
    __syncthreads();
    sG[m] = sbp[m + 1] - sa[m] * sbp[0];
    sGh[m] = -sa[m];   // input vector of the all-pole filter (b = [1])
    const size_t rec = backward ? (bt.bwd_stride ? (size_t)bt.bwd_stride : Tab::bwd_rec(f64))
                                : (bt.fwd_stride ? (size_t)bt.fwd_stride : Tab::fwd_rec(f64));
    char *R = (backward ? bwd_tabs : fwd_tabs) + (size_t)ch * rec;
    __syncthreads();

    if (!backward) {
        float *g = reinterpret_cast<float *>(R + Tab::F_G);
        float *RL = reinterpret_cast<float *>(R + Tab::F_RL);
        float *OL = reinterpret_cast<float *>(R + Tab::F_OL);
        double v[MB];
#pragma unroll
        for (int k = 0; k < MB; ++k) v[k] = k == m ? 1.0 : 0.0;
        for (int i = 0; i < L; ++i) {
            OL[i * MB + m] = (float)v[0];
            sOL[i][m] = v[0];
#pragma unroll
            for (int k = 0; k < MB; ++k) sX[k][m] = v[k];
            __syncthreads();
            // R_L[:, L-1-i] = F^i Gv: component m = sum_j X[m][j] Gv_j
            double acc = 0.0;
#pragma unroll 8
            for (int j = 0; j < MB; ++j) acc += sX[m][j] * sG[j];
            RL[m * L + (L - 1 - i)] = (float)acc;
            __syncthreads();
            const double v0 = v[0];
#pragma unroll
            for (int k = 0; k < MB; ++k) v[k] = (k + 1 < MB ? v[k + 1] : 0.0) - sa[k] * v0;
        }
#pragma unroll
        for (int k = 0; k < MB; ++k) sA[k][m] = v[k];
        // g[0] = b0, g[n] = e1^T F^(n-1) Gv = sum_j O_L[n-1][j] Gv_j
        for (int n = m; n < L; n += MB) {
            double acc = 0.0;
            if (n == 0) {
                acc = sbp[0];
            } else {
                for (int j = 0; j < MB; ++j) acc += sOL[n - 1][j] * sG[j];
            }
            g[n] = (float)acc;
        }
    } else {
        float *g = reinterpret_cast<float *>(R + Tab::B_G);
        float *h = reinterpret_cast<float *>(R + Tab::B_H);
        float *Ou = reinterpret_cast<float *>(R + Tab::B_OU);
        float *Ogx = reinterpret_cast<float *>(R + Tab::B_OGX);
        float *C = reinterpret_cast<float *>(R + Tab::b_coef(f64));
        C[m] = (float)sa[m];
        C[MB + m] = (float)sbp[m];
        if (m == 0) C[2 * MB] = (float)sbp[MB];
        // first rows of F^i for g and h
        double v[MB];
#pragma unroll
        for (int k = 0; k < MB; ++k) v[k] = k == m ? 1.0 : 0.0;
        float *OLb = reinterpret_cast<float *>(R + Tab::b_ol(f64));
        for (int i = 0; i < L; ++i) {
            sOL[i][m] = v[0];
            OLb[i * MB + m] = (float)v[0];
            const double v0 = v[0];
#pragma unroll
            for (int k = 0; k < MB; ++k) v[k] = (k + 1 < MB ? v[k + 1] : 0.0) - sa[k] * v0;
        }
        __syncthreads();
        for (int n = m; n < L; n += MB) {
            double ag = 0.0, ah = 0.0;
            if (n == 0) {
                ag = sbp[0];
                ah = 1.0;
            } else {
                for (int j = 0; j < MB; ++j) {
                    ag += sOL[n - 1][j] * sG[j];
                    ah += sOL[n - 1][j] * sGh[j];
                }
            }
            g[n] = (float)ag;
            h[n] = (float)ah;
        }
        // column m of O^u (anti-causal recursion from u[L+m] = 1), O^gx on the fly
        double e[MB + 1];
#pragma unroll
        for (int j = 0; j <= MB; ++j) e[j] = 0.0;
#pragma unroll
        for (int j = 0; j < MB; ++j) e[j + 1] = j == m ? 1.0 : 0.0;
        for (int n = L - 1; n >= 0; --n) {
            double un = 0.0;
#pragma unroll
            for (int k = 1; k <= MB; ++k) un -= sa[k - 1] * e[k];
            e[0] = un;
            double gxn = 0.0;
#pragma unroll
            for (int k = 0; k <= MB; ++k) gxn += sbp[k] * e[k];
            Ou[n * MB + m] = (float)un;
            Ogx[n * MB + m] = (float)gxn;
            if (n < MB) sA[n][m] = un;
#pragma unroll
            for (int j = MB; j > 0; --j) e[j] = e[j - 1];
        }
    }
    __syncthreads();
    char *S = R + (backward ? Tab::B_SCAN : Tab::F_SCAN);
    if (f64) {
        float2 *At = reinterpret_cast<float2 *>(S);   // double words (hi, lo), column-major
        for (int j = 0; j < MB; ++j) {
            const double v = sA[m][j];
            const float hi = (float)v;
            At[j * MB + m] = make_float2(hi, (float)(v - (double)hi));
        }
        if constexpr (Tab::kBlockScan) {   // then A^4, by squaring twice in FP64
            for (int sq = 0; sq < 2; ++sq) {
                double row[MB];
                for (int j = 0; j < MB; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < MB; ++k) acc += sA[m][k] * sA[k][j];
                    row[j] = acc;
                }
                __syncthreads();
                for (int j = 0; j < MB; ++j) sA[m][j] = row[j];
                __syncthreads();
            }
            for (int j = 0; j < MB; ++j) {
                const double v = sA[m][j];
                const float hi = (float)v;
                At[MB * MB + j * MB + m] = make_float2(hi, (float)(v - (double)hi));
            }
        }
    } else {
        float *P = reinterpret_cast<float *>(S);
        for (int kp = 0; kp < Tab::NPOW; ++kp) {
            for (int j = 0; j < MB; ++j) P[(kp * MB + m) * MB + j] = (float)sA[m][j];
            if (kp + 1 == Tab::NPOW) break;
            double row[MB];
            for (int j = 0; j < MB; ++j) {
                double acc = 0.0;
                for (int k = 0; k < MB; ++k) acc += sA[m][k] * sA[k][j];
                row[j] = acc;
            }
            __syncthreads();
            for (int j = 0; j < MB; ++j) sA[m][j] = row[j];
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Higher orders (MB >= 8) with the double-word scan: both records of a channel per
// block, every table entry a short FP64 sum over the impulse responses h (of 1/A) and
// g (of B/A), rounded to FP32 (the scan blocks to (hi, lo) float pairs).  Closed forms
// need O(M) multiply-adds per entry where stepping the TDF-II transition L times costs
// O(L M) per column, so FP64 stays affordable on GB300's narrow FP64 pipe (double words
// lose digits here: the sums cancel by orders of magnitude for high-order filters).
// With the TDF-II state s_k[n] = sum_{l>k} (b_l x[n+k-l] - a_l y[n+k-l]) and the state
// e_m equivalent to injecting 1 at time m (so its free response is h[n - m]):
//   O_L[i][m] = h[i - m]                      R_L[m][j] = b_{L+m-j} - sum_{l>m} a_l g[L+m-l-j]
//   Abar(K)[k][m] = -sum_{l>k} a_l h[K + k - l - m]        (K = L, and 4L for Abar^4)
//   O^u(K)[n][m] = -sum_{p=0..M-1-m} a_{p+1+m} h[K - 1 - n - p]
//       (the anti-causal free response from u[K + m] = 1; Abar' = O^u(L)[0:MB, :],
//        Abar'^4 = O^u(4L)[0:MB, :])
//   O^gx[n][m] = sum_k b_k U(n + k, m),  U(t, m) = O^u[t][m] (t < L), [t - L == m] (t >= L)
// (terms past the channel's orders are zero; b_{L+m-j} only where 0 < L+m-j-m <= N).
// Checked against the step-by-step construction, which these replace, to 1e-15.
// ---------------------------------------------------------------------------
template <int MB>
struct HiSetupSmem {
    static constexpr int H = ChunkTab<MB>::kBlockScan ? 4 * kL + MB : kL + MB;   // h[0 .. H)
    static constexpr int G = kL + MB;                                           // g[0 .. G)
    double h[H], g[G];
    double ou[kL * MB];   // O^u(L)[n][m], row-major
    double a[MB], b[MB + 1];
};

template <int MB>
__global__ void __launch_bounds__(128) setup_hi_kernel(const float *__restrict__ b,
                                                       const float *__restrict__ a,
                                                       char *__restrict__ fwd_tabs,
                                                       char *__restrict__ bwd_tabs,
                                                       unsigned long long *__restrict__ counter,
                                                       Batch bt) {
    using Tab = ChunkTab<MB>;
    using SM = HiSetupSmem<MB>;
    constexpr int NT = 128;
    extern __shared__ float4 smem4[];
    SM &sm = *reinterpret_cast<SM *>(smem4);
    const int t = threadIdx.x, lane = t & 31;
    if (counter && blockIdx.x == 0 && t == 0) *counter = 0ull;
    int64_t ch;
    if (!work_channel(bt, (int64_t)blockIdx.x, &ch)) return;   // uniform across the block
    const Channel c = channel_of(bt, ch);
    for (int k = t; k < MB; k += NT) sm.a[k] = k < c.M ? (double)a[ch * bt.Mstride + k] : 0.0;
    for (int k = t; k <= MB; k += NT) sm.b[k] = k <= c.N ? (double)b[ch * bt.Nstride + k] : 0.0;
    __syncthreads();
    const int M = c.M < MB ? c.M : MB;
    // h by the all-pole difference equation (warp 0, the lanes share each step's sum)
    if (t < 32) {
        if (t == 0) sm.h[0] = 1.0;
        __syncwarp();
        for (int n = 1; n < SM::H; ++n) {
            double acc = 0.0;
            for (int j = lane + 1; j <= M; j += 32)
                if (j <= n) acc = fma(-sm.a[j - 1], sm.h[n - j], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) sm.h[n] = acc;
            __syncwarp();
        }
    }
    __syncthreads();
    auto H = [&](int n) { return n >= 0 ? sm.h[n] : 0.0; };
    // g = b * h
    for (int n = t; n < SM::G; n += NT) {
        double acc = 0.0;
        for (int k = 0; k <= c.N && k <= n; ++k) acc = fma(sm.b[k], sm.h[n - k], acc);
        sm.g[n] = acc;
    }
    // O^u(L) into shared memory
    for (int e = t; e < kL * MB; e += NT) {
        const int n = e / MB, m = e % MB;
        double acc = 0.0;
        for (int p = 0; p + 1 + m <= M; ++p) acc = fma(-sm.a[p + m], H(kL - 1 - n - p), acc);
        sm.ou[e] = acc;
    }
    __syncthreads();
    auto Gf = [&](int n) { return n >= 0 ? sm.g[n] : 0.0; };
    auto abar = [&](int K, int k, int m) {   // Abar(K)[k][m]
        double acc = 0.0;
        for (int l = k + 1; l <= M; ++l) acc = fma(-sm.a[l - 1], H(K + k - l - m), acc);
        return acc;
    };
    auto ou4 = [&](int n, int m) {            // O^u(4L)[n][m]
        double acc = 0.0;
        for (int p = 0; p + 1 + m <= M; ++p) acc = fma(-sm.a[p + m], H(4 * kL - 1 - n - p), acc);
        return acc;
    };
    auto pair = [](double v) {                // (hi, lo) float pair of v
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    };
    if (fwd_tabs) {
        char *R = fwd_tabs + (size_t)ch * (bt.fwd_stride ? (size_t)bt.fwd_stride : Tab::fwd_rec(true));
        float *g = reinterpret_cast<float *>(R + Tab::F_G);
        float *RL = reinterpret_cast<float *>(R + Tab::F_RL);
        float *OL = reinterpret_cast<float *>(R + Tab::F_OL);
        for (int n = t; n < kL; n += NT) g[n] = (float)sm.g[n];
        for (int e = t; e < MB * kL; e += NT) {
            const int m = e / kL, j = e % kL;
            const int lb = kL + m - j;   // the b term's index
            double acc = (lb > m && lb <= c.N) ? sm.b[lb] : 0.0;
            for (int l = m + 1; l <= M; ++l) acc = fma(-sm.a[l - 1], Gf(kL + m - l - j), acc);
            RL[e] = (float)acc;
        }
        for (int e = t; e < kL * MB; e += NT) {
            const int i = e / MB, m = e % MB;
            OL[e] = (float)H(i - m);
        }
        float2 *At = reinterpret_cast<float2 *>(R + Tab::F_SCAN);   // column-major
        for (int e = t; e < MB * MB; e += NT) {
            const int j = e / MB, m = e % MB;   // At[j * MB + m] = Abar[m][j]
            At[e] = pair(abar(kL, m, j));
            if constexpr (Tab::kBlockScan) At[MB * MB + e] = pair(abar(4 * kL, m, j));
        }
    }
    if (bwd_tabs) {
        char *R = bwd_tabs + (size_t)ch * (bt.bwd_stride ? (size_t)bt.bwd_stride : Tab::bwd_rec(true));
        float *g = reinterpret_cast<float *>(R + Tab::B_G);
        float *hv = reinterpret_cast<float *>(R + Tab::B_H);
        float *Ou = reinterpret_cast<float *>(R + Tab::B_OU);
        float *Ogx = reinterpret_cast<float *>(R + Tab::B_OGX);
        for (int n = t; n < kL; n += NT) {
            g[n] = (float)sm.g[n];
            hv[n] = (float)sm.h[n];
        }
        for (int e = t; e < kL * MB; e += NT) {
            const int n = e / MB, m = e % MB;
            Ou[e] = (float)sm.ou[e];
            double acc = 0.0;
            for (int k = 0; k <= c.N; ++k) {
                const int tt = n + k;
                if (tt < kL) acc = fma(sm.b[k], sm.ou[tt * MB + m], acc);
                else if (tt - kL == m) acc += sm.b[k];
            }
            Ogx[e] = (float)acc;
        }
        float2 *At = reinterpret_cast<float2 *>(R + Tab::B_SCAN);   // column-major
        for (int e = t; e < MB * MB; e += NT) {
            const int j = e / MB, m = e % MB;   // At[j * MB + m] = Abar'[m][j] = O^u[m][j]
            At[e] = pair(sm.ou[m * MB + j]);
            if constexpr (Tab::kBlockScan) At[MB * MB + e] = pair(ou4(m, j));
        }
        float *C = reinterpret_cast<float *>(R + Tab::b_coef(true));
        for (int k = t; k < MB; k += NT) C[k] = (float)sm.a[k];
        for (int k = t; k <= MB; k += NT) C[MB + k] = (float)sm.b[k];
        if constexpr (MB > 4) {
            float *OLb = reinterpret_cast<float *>(R + Tab::b_ol(true));
            for (int e = t; e < kL * MB; e += NT) {
                const int i = e / MB, m = e % MB;
                OLb[e] = (float)H(i - m);
            }
        }
    }
}

}  // namespace

cudaError_t launch_chunk_setup(const float *b, const float *a, char *fwd_tabs, char *bwd_tabs,
                               unsigned long long *counter, const Batch &bt, int MB,
                               bool fp64_scan, cudaStream_t st) {
    if (!fwd_tabs && !bwd_tabs) return cudaErrorInvalidValue;
    const unsigned gy = (fwd_tabs && bwd_tabs) ? 2u : 1u;
    const dim3 small_grid((unsigned)((bt.B + kSmallWarps - 1) / kSmallWarps), 1);   // both records per warp
    const dim3 large_grid((unsigned)bt.B, gy);
    auto small = [&](auto kern) -> cudaError_t {
        kern<<<small_grid, 32 * kSmallWarps, 0, st>>>(b, a, fwd_tabs, bwd_tabs, counter, bt, fp64_scan); note_launch();
        return cudaGetLastError();
    };
    auto large = [&](auto kern, int mb, size_t smem) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<large_grid, mb, smem, st>>>(b, a, fwd_tabs, bwd_tabs, counter, bt, fp64_scan); note_launch();
        return cudaGetLastError();
    };
    auto hi = [&](auto kern, size_t smem) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<(unsigned)bt.B, 128, smem, st>>>(b, a, fwd_tabs, bwd_tabs, counter, bt); note_launch();
        return cudaGetLastError();
    };
    if (fp64_scan) {
        switch (MB) {
            case 8: return hi(setup_hi_kernel<8>, sizeof(HiSetupSmem<8>));
            case 16: return hi(setup_hi_kernel<16>, sizeof(HiSetupSmem<16>));
            case 32: return hi(setup_hi_kernel<32>, sizeof(HiSetupSmem<32>));
            case 64: return hi(setup_hi_kernel<64>, sizeof(HiSetupSmem<64>));
            default: break;
        }
    }
    switch (MB) {
        case 2: return small(setup_small_kernel<2>);
        case 4: return small(setup_small_kernel<4>);
        case 8: return large(setup_large_kernel<8>, 8, setup_large_smem<8>());
        case 16: return large(setup_large_kernel<16>, 16, setup_large_smem<16>());
        case 32: return large(setup_large_kernel<32>, 32, setup_large_smem<32>());
        case 64: return large(setup_large_kernel<64>, 64, setup_large_smem<64>());
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dfilt
