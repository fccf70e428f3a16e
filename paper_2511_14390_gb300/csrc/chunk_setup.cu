// Coefficient setup of the chunked algorithm: per channel, in FP64, the impulse
// responses, the free-response and end-state blocks, and the chunk transition of the
// chunk algebra (see chunk.cuh).  FP64 because companion-matrix powers of high-order
// filters grow transiently by orders of magnitude before they decay; the transition
// is formed by L successive companion products (no repeated squaring, which loses
// accuracy on those filters).
//
// GB300's FP64 pipe is narrow and a warp-wide FP64 instruction costs it the same
// whether 1 or 32 lanes are active, so both variants keep every lane busy:
//   * low orders (MB <= 4): one channel per thread, everything in registers, in
//     double-word arithmetic (dword.cuh) on the full-rate FP32 pipes;
//   * higher orders: one block per channel, thread m evolves column m of F^i
//     (i = 0..L) and every table is read off those columns in parallel:
//       O_L[i][m] = (F^i e_m)[0],  g[n] = sum_m Gv_m O_L[n-1][m] (n >= 1),
//       h[n] likewise with the all-pole input vector, R_L[:, L-1-i] = F^i Gv
//       (a reduction over the columns held in shared memory), Abar = F^L.
//     The backward's O^u columns run the anti-causal all-pole recursion from a
//     unit future state, one column per thread.
#include "chunk.cuh"
#include "dword.cuh"

namespace dfilt {

namespace {

// ---------------------------------------------------------------------------
// low orders: one channel per thread, double-word arithmetic on the FP32 pipes
// ---------------------------------------------------------------------------
template <int MB>
__global__ void __launch_bounds__(64) setup_small_kernel(const float *__restrict__ b,
                                                         const float *__restrict__ a,
                                                         char *__restrict__ ws, Batch bt,
                                                         bool f64, bool backward) {
    using Tab = ChunkTab<MB>;
    constexpr int L = kL;
    const int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ch == 0) *reinterpret_cast<unsigned long long *>(ws) = 0ull;   // work counter
    if (ch >= bt.B) return;
    const Channel c = channel_of(bt, ch);
    dw av[MB], bp[MB + 1], G[MB];
#pragma unroll
    for (int k = 0; k < MB; ++k) av[k] = dw_make(k < c.M ? a[ch * bt.Mstride + k] : 0.f);
#pragma unroll
    for (int k = 0; k <= MB; ++k) bp[k] = dw_make(k <= c.N ? b[ch * bt.Nstride + k] : 0.f);
#pragma unroll
    for (int k = 0; k < MB; ++k) G[k] = bp[k + 1] - av[k] * bp[0];
    const size_t rec = backward ? Tab::bwd_rec(f64) : Tab::fwd_rec(f64);
    char *R = ws + kWsHeader + (size_t)ch * rec;
    dw A[MB][MB];   // chunk transition
    if (!backward) {
        float *g = reinterpret_cast<float *>(R + Tab::F_G);
        float *RL = reinterpret_cast<float *>(R + Tab::F_RL);
        float *OL = reinterpret_cast<float *>(R + Tab::F_OL);
        // r = e1^T F^i (rows of O_L), v = F^i Gv (columns of R_L, g[i+1] = v_0)
        dw r[MB], v[MB];
#pragma unroll
        for (int k = 0; k < MB; ++k) {
            r[k] = dw_make(k == 0 ? 1.f : 0.f);
            v[k] = G[k];
        }
        // rows[j] = e1^T F^(L-j), j = 0..MB, for the rows of Abar = F^L (below)
        dw rows[MB + 1][MB];
        g[0] = dw_to_float(bp[0]);
        for (int i = 0; i < L; ++i) {
#pragma unroll
            for (int m = 0; m < MB; ++m) OL[i * MB + m] = dw_to_float(r[m]);
            if (i + 1 < L) g[i + 1] = dw_to_float(v[0]);
#pragma unroll
            for (int k = 0; k < MB; ++k) RL[k * L + (L - 1 - i)] = dw_to_float(v[k]);
#pragma unroll
            for (int j = 1; j <= MB; ++j)
                if (i == L - j) {
#pragma unroll
                    for (int k = 0; k < MB; ++k) rows[j][k] = r[k];
                }
            // (F v)_k = v_{k+1} - a_{k+1} v_0 ;  (r F)_0 = -sum_k r_k a_{k+1}, (r F)_j = r_{j-1}
            const dw v0 = v[0];
#pragma unroll
            for (int k = 0; k < MB; ++k) v[k] = (k + 1 < MB ? v[k + 1] : dw_make(0.f)) - av[k] * v0;
            dw r0 = dw_make(0.f);
#pragma unroll
            for (int k = 0; k < MB; ++k) r0 = r0 - r[k] * av[k];
#pragma unroll
            for (int k = MB - 1; k > 0; --k) r[k] = r[k - 1];
            r[0] = r0;
        }
#pragma unroll
        for (int k = 0; k < MB; ++k) rows[0][k] = r[k];
        // Rows of F^L from e_k^T F = -a_{k+1} e_0^T + e_{k+1}^T:
        //   e_k^T F^L = -sum_{j=0}^{MB-1-k} a_{k+1+j} e_0^T F^(L-1-j)   (k >= 1)
#pragma unroll
        for (int m = 0; m < MB; ++m) A[0][m] = rows[0][m];
#pragma unroll
        for (int k = 1; k < MB; ++k)
#pragma unroll
            for (int m = 0; m < MB; ++m) {
                dw acc = dw_make(0.f);
#pragma unroll
                for (int j = 0; j <= MB - 1 - k; ++j) acc = acc - av[k + j] * rows[1 + j][m];
                A[k][m] = acc;
            }
    } else {
        float *g = reinterpret_cast<float *>(R + Tab::B_G);
        float *h = reinterpret_cast<float *>(R + Tab::B_H);
        float *Ou = reinterpret_cast<float *>(R + Tab::B_OU);
        float *Ogx = reinterpret_cast<float *>(R + Tab::B_OGX);
        // impulse responses by the difference equation, sliding windows of MB outputs
        dw wg[MB], wh[MB];
#pragma unroll
        for (int k = 0; k < MB; ++k) wg[k] = wh[k] = dw_make(0.f);
        for (int n = 0; n < L; ++n) {
            dw yg = dw_make(0.f), yh = dw_make(n == 0 ? 1.f : 0.f);
#pragma unroll
            for (int k = 0; k <= MB; ++k)
                if (n == k) yg = bp[k];   // numerator input b_n (zero past order MB)
#pragma unroll
            for (int k = 0; k < MB; ++k) {
                yg = yg - av[k] * wg[k];
                yh = yh - av[k] * wh[k];
            }
#pragma unroll
            for (int k = MB - 1; k > 0; --k) {
                wg[k] = wg[k - 1];
                wh[k] = wh[k - 1];
            }
            wg[0] = yg;
            wh[0] = yh;
            g[n] = dw_to_float(yg);
            h[n] = dw_to_float(yh);
        }
        // O^u and O^gx columns: anti-causal all-pole recursion from u[L+m] = delta
#pragma unroll
        for (int m = 0; m < MB; ++m) {
            dw e[MB + 1];   // e[j] = u[n + j], j = 0..MB
#pragma unroll
            for (int j = 0; j <= MB; ++j) e[j] = dw_make(j == m + 1 ? 1.f : 0.f);
            for (int n = L - 1; n >= 0; --n) {
                dw un = dw_make(0.f);
#pragma unroll
                for (int k = 1; k <= MB; ++k) un = un - av[k - 1] * e[k];
                e[0] = un;
                dw gxn = dw_make(0.f);
#pragma unroll
                for (int k = 0; k <= MB; ++k) gxn = gxn + bp[k] * e[k];
                Ou[n * MB + m] = dw_to_float(un);
                Ogx[n * MB + m] = dw_to_float(gxn);
#pragma unroll
                for (int k = 0; k < MB; ++k)
                    if (n == k) A[k][m] = un;
#pragma unroll
                for (int j = MB; j > 0; --j) e[j] = e[j - 1];
            }
        }
    }
    char *S = R + (backward ? Tab::B_SCAN : Tab::F_SCAN);
    if (f64) {
        double *At = reinterpret_cast<double *>(S);
#pragma unroll
        for (int j = 0; j < MB; ++j)
#pragma unroll
            for (int m = 0; m < MB; ++m) At[j * MB + m] = dw_to_double(A[m][j]);
    } else {
        float *P = reinterpret_cast<float *>(S);
        for (int kp = 0; kp < Tab::NPOW; ++kp) {
#pragma unroll
            for (int i = 0; i < MB; ++i)
#pragma unroll
                for (int j = 0; j < MB; ++j) P[(kp * MB + i) * MB + j] = dw_to_float(A[i][j]);
            if (kp + 1 == Tab::NPOW) break;
            dw Q[MB][MB];
#pragma unroll
            for (int i = 0; i < MB; ++i)
#pragma unroll
                for (int j = 0; j < MB; ++j) {
                    dw acc = dw_make(0.f);
#pragma unroll
                    for (int k = 0; k < MB; ++k) acc = acc + A[i][k] * A[k][j];
                    Q[i][j] = acc;
                }
#pragma unroll
            for (int i = 0; i < MB; ++i)
#pragma unroll
                for (int j = 0; j < MB; ++j) A[i][j] = Q[i][j];
        }
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
__global__ void __launch_bounds__(MB) setup_large_kernel(const float *__restrict__ b,
                                                         const float *__restrict__ a,
                                                         char *__restrict__ ws, Batch bt,
                                                         bool f64, bool backward) {
    using Tab = ChunkTab<MB>;
    constexpr int L = kL;
    extern __shared__ double sdyn[];
    double *sa = sdyn, *sbp = sa + MB, *sG = sbp + MB + 1, *sGh = sG + MB;
    // columns of F^i at the current step (row k, col m), the transition, first rows
    double(*sX)[MB + 1] = reinterpret_cast<double(*)[MB + 1]>(sGh + MB);
    double(*sA)[MB + 1] = sX + MB;
    double(*sOL)[MB + 1] = sA + MB;

    const int64_t ch = blockIdx.x;
    const int m = threadIdx.x;
    if (ch == 0 && m == 0) *reinterpret_cast<unsigned long long *>(ws) = 0ull;
    const Channel c = channel_of(bt, ch);
    sa[m] = m < c.M ? (double)a[ch * bt.Mstride + m] : 0.0;
    sbp[m] = m <= c.N ? (double)b[ch * bt.Nstride + m] : 0.0;
    if (m == 0) sbp[MB] = MB <= c.N ? (double)b[ch * bt.Nstride + MB] : 0.0;
    __syncthreads();
    sG[m] = sbp[m + 1] - sa[m] * sbp[0];
    sGh[m] = -sa[m];   // input vector of the all-pole filter (b = [1])
    const size_t rec = backward ? Tab::bwd_rec(f64) : Tab::fwd_rec(f64);
    char *R = ws + kWsHeader + (size_t)ch * rec;
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
        // first rows of F^i for g and h
        double v[MB];
#pragma unroll
        for (int k = 0; k < MB; ++k) v[k] = k == m ? 1.0 : 0.0;
        for (int i = 0; i < L; ++i) {
            sOL[i][m] = v[0];
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
        double *At = reinterpret_cast<double *>(S);
        for (int j = 0; j < MB; ++j) At[j * MB + m] = sA[m][j];
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

}  // namespace

cudaError_t launch_chunk_setup(const float *b, const float *a, void *ws, const Batch &bt, int MB,
                               bool fp64_scan, bool backward, cudaStream_t st) {
    char *w = static_cast<char *>(ws);
    const unsigned small_grid = (unsigned)((bt.B + 63) / 64);
    const unsigned large_grid = (unsigned)bt.B;
    auto large = [&](auto kern, int mb, size_t smem) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<large_grid, mb, smem, st>>>(b, a, w, bt, fp64_scan, backward);
        return cudaGetLastError();
    };
    switch (MB) {
        case 2: setup_small_kernel<2><<<small_grid, 64, 0, st>>>(b, a, w, bt, fp64_scan, backward); break;
        case 4: setup_small_kernel<4><<<small_grid, 64, 0, st>>>(b, a, w, bt, fp64_scan, backward); break;
        case 8: return large(setup_large_kernel<8>, 8, setup_large_smem<8>());
        case 16: return large(setup_large_kernel<16>, 16, setup_large_smem<16>());
        case 32: return large(setup_large_kernel<32>, 32, setup_large_smem<32>());
        case 64: return large(setup_large_kernel<64>, 64, setup_large_smem<64>());
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dfilt
