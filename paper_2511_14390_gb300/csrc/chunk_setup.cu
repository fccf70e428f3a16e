// Coefficient setup of the chunked algorithm: per channel, in FP64, the impulse
// responses, the free-response and end-state blocks, and the chunk transition of the
// chunk algebra (see chunk.cuh).  FP64 because companion-matrix powers of high-order
// filters grow transiently by orders of magnitude before they decay; the transition
// is formed by L successive companion products (no repeated squaring, which loses
// accuracy on those filters).  One block per channel; the serial chains run on
// separate threads in parallel.
#include "chunk.cuh"

namespace dfilt {

namespace {

template <int MB>
__global__ void __launch_bounds__(128) chunk_setup_kernel(const float *__restrict__ b,
                                                          const float *__restrict__ a,
                                                          char *__restrict__ ws, Batch bt,
                                                          bool f64, bool backward) {
    using Tab = ChunkTab<MB>;
    constexpr int L = kL;
    __shared__ double sa[MB], sbp[MB + 1], sG[MB];
    __shared__ double sA[MB][MB + 1];     // transition (row-major, padded)
    __shared__ double sP[MB][MB + 1];     // squaring scratch

    const int64_t ch = blockIdx.x;
    const int tid = threadIdx.x;
    if (ch == 0 && tid == 0) *reinterpret_cast<unsigned long long *>(ws) = 0ull;   // work counter
    const Channel c = channel_of(bt, ch);
    for (int k = tid; k < MB; k += blockDim.x) sa[k] = k < c.M ? (double)a[ch * bt.Mstride + k] : 0.0;
    for (int k = tid; k <= MB; k += blockDim.x) sbp[k] = k <= c.N ? (double)b[ch * bt.Nstride + k] : 0.0;
    __syncthreads();
    for (int k = tid; k < MB; k += blockDim.x) sG[k] = sbp[k + 1] - sa[k] * sbp[0];
    __syncthreads();

    const size_t rec = backward ? Tab::bwd_rec(f64) : Tab::fwd_rec(f64);
    char *R = ws + kWsHeader + (size_t)ch * rec;

    if (!backward) {
        float *g = reinterpret_cast<float *>(R + Tab::F_G);
        float *RL = reinterpret_cast<float *>(R + Tab::F_RL);
        float *OL = reinterpret_cast<float *>(R + Tab::F_OL);
        if (tid == 64) {
            // g[0] = b0, g[n] = e1^T F^(n-1) Gv
            double v[MB];
            for (int k = 0; k < MB; ++k) v[k] = sG[k];
            g[0] = (float)sbp[0];
            for (int n = 1; n < L; ++n) {
                g[n] = (float)v[0];
                const double v0 = v[0];
                for (int k = 0; k < MB; ++k) v[k] = (k + 1 < MB ? v[k + 1] : 0.0) - sa[k] * v0;
            }
        } else if (tid == 65) {
            // R_L[:, j] = F^(L-1-j) Gv
            double v[MB];
            for (int k = 0; k < MB; ++k) v[k] = sG[k];
            for (int j = L - 1; j >= 0; --j) {
                for (int k = 0; k < MB; ++k) RL[k * L + j] = (float)v[k];
                const double v0 = v[0];
                for (int k = 0; k < MB; ++k) v[k] = (k + 1 < MB ? v[k + 1] : 0.0) - sa[k] * v0;
            }
        } else if (tid == 66) {
            // O_L[i] = e1^T F^i:  (r F)_0 = -sum_k r_k a_{k+1},  (r F)_j = r_{j-1}
            double r[MB];
            for (int k = 0; k < MB; ++k) r[k] = k == 0 ? 1.0 : 0.0;
            for (int i = 0; i < L; ++i) {
                for (int k = 0; k < MB; ++k) OL[i * MB + k] = (float)r[k];
                double r0 = 0.0;
                for (int k = 0; k < MB; ++k) r0 -= r[k] * sa[k];
                for (int k = MB - 1; k > 0; --k) r[k] = r[k - 1];
                r[0] = r0;
            }
        } else if (tid < MB) {
            // column tid of Abar = F^L by L companion products
            double v[MB];
            for (int k = 0; k < MB; ++k) v[k] = k == tid ? 1.0 : 0.0;
            for (int n = 0; n < L; ++n) {
                const double v0 = v[0];
                for (int k = 0; k < MB; ++k) v[k] = (k + 1 < MB ? v[k + 1] : 0.0) - sa[k] * v0;
            }
            for (int k = 0; k < MB; ++k) sA[k][tid] = v[k];
        }
    } else {
        float *g = reinterpret_cast<float *>(R + Tab::B_G);
        float *h = reinterpret_cast<float *>(R + Tab::B_H);
        float *Ou = reinterpret_cast<float *>(R + Tab::B_OU);
        float *Ogx = reinterpret_cast<float *>(R + Tab::B_OGX);
        if (tid == 64 || tid == 65) {
            // impulse responses of B/A (tid 64) and 1/A (tid 65) by the difference equation
            const bool num = tid == 64;
            double yv[L];
            for (int n = 0; n < L; ++n) {
                double acc = num ? (n <= MB ? sbp[n] : 0.0) : (n == 0 ? 1.0 : 0.0);
                for (int k = 1; k <= MB && k <= n; ++k) acc -= sa[k - 1] * yv[n - k];
                yv[n] = acc;
                (num ? g : h)[n] = (float)acc;
            }
        } else if (tid < MB) {
            // column tid of O^u: anti-causal all-pole recursion from u[L + m] = delta(m, tid)
            double e[L + MB];
            for (int k = 0; k < MB; ++k) e[L + k] = k == tid ? 1.0 : 0.0;
            for (int n = L - 1; n >= 0; --n) {
                double acc = 0.0;
                for (int k = 1; k <= MB; ++k) acc -= sa[k - 1] * e[n + k];
                e[n] = acc;
            }
            for (int n = 0; n < L; ++n) Ou[n * MB + tid] = (float)e[n];
            for (int n = 0; n < MB; ++n) sA[n][tid] = e[n];   // Abar' = O^u[0:MB, :]
            // O^gx[i][tid] = sum_k b_k u[i+k] over the extended column
            for (int i = 0; i < L; ++i) {
                double acc = 0.0;
                for (int k = 0; k <= MB; ++k) acc += sbp[k] * e[i + k];
                Ogx[i * MB + tid] = (float)acc;
            }
        }
    }
    __syncthreads();

    char *S = R + (backward ? Tab::B_SCAN : Tab::F_SCAN);
    if (f64) {
        double *At = reinterpret_cast<double *>(S);
        for (int idx = tid; idx < MB * MB; idx += blockDim.x) {
            const int m = idx % MB, j = idx / MB;
            At[j * MB + m] = sA[m][j];
        }
    } else {
        float *P = reinterpret_cast<float *>(S);
        for (int kp = 0; kp < Tab::NPOW; ++kp) {
            for (int idx = tid; idx < MB * MB; idx += blockDim.x)
                P[(size_t)kp * MB * MB + idx] = (float)sA[idx / MB][idx % MB];
            if (kp + 1 == Tab::NPOW) break;
            for (int idx = tid; idx < MB * MB; idx += blockDim.x) {
                const int i = idx / MB, j = idx % MB;
                double acc = 0.0;
                for (int k = 0; k < MB; ++k) acc += sA[i][k] * sA[k][j];
                sP[i][j] = acc;
            }
            __syncthreads();
            for (int idx = tid; idx < MB * MB; idx += blockDim.x) sA[idx / MB][idx % MB] = sP[idx / MB][idx % MB];
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_chunk_setup(const float *b, const float *a, void *ws, const Batch &bt, int MB,
                               bool fp64_scan, bool backward, cudaStream_t st) {
    const dim3 grid((unsigned)bt.B), block(128);
    char *w = static_cast<char *>(ws);
    switch (MB) {
#define X(V)                                                                                       \
    case V:                                                                                        \
        chunk_setup_kernel<V><<<grid, block, 0, st>>>(b, a, w, bt, fp64_scan, backward);           \
        break;
        X(2) X(4) X(8) X(16) X(32) X(64)
#undef X
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dfilt
