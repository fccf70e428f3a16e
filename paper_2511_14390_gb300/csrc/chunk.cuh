// Per-channel table layout of the chunked algorithm, shared by the setup kernels and
// the forward/backward tensor-core kernels.
//
// Chunk algebra (Sec. 3.2's associative operator applied at chunk granularity,
// chunk length L = 64, TDF-II state of dimension MB, M padded with zeros):
//   forward   Y_c = T_g X_c + O_L S_c,    S_{c+1} = Abar S_c + R_L X_c,   S_0 = zi
//   backward  U_c = T_h^a G_c + O^u S'_c, GX_c = T_g^a G_c + O^gx S'_c,   S'_{c-1} = U_c[0:MB]
// where g / h are the impulse responses of B/A and 1/A, Abar = F^L (F the TDF-II
// transition), O_L[i] = e_1^T F^i, R_L[:, j] = F^(L-1-j) Gv, and S'_c holds the next
// MB adjoint values u[(c+1)L ..] (zero past the end, App. A).  Backward transition
// Abar' = O^u[0:MB, :].
#pragma once

#include "kernels.h"

namespace dfilt {

template <int MB>
struct ChunkTab {
    // padded width of the state block inside the tensor-core B operand
    static constexpr int MPAD = MB <= 16 ? 16 : (MB <= 32 ? 32 : 64);
    static constexpr int NFWD = kL + MPAD;          // forward MMA N: [T_g rows | R_L rows]
    static constexpr int NBWD = 2 * kL;             // backward MMA N: [T_g^a rows | T_h^a rows]
    static constexpr int NPOW = 6;                  // Abar^(2^k), k < 6 (warp scan + carries)

    // forward record (bytes): g[L] f32 | RL[MB][L] f32 | OL[L][MB] f32 | scan block
    static constexpr size_t F_G = 0;
    static constexpr size_t F_RL = F_G + kL * 4;
    static constexpr size_t F_OL = F_RL + (size_t)MB * kL * 4;
    static constexpr size_t F_SCAN = (F_OL + (size_t)kL * MB * 4 + 15) / 16 * 16;
    // backward record: g[L] | h[L] | Ou[L][MB] | Ogx[L][MB] | scan block | coefficients
    // (a_1..a_MB, b_0..b_MB as f32, zero past the channel's orders)
    static constexpr size_t B_G = 0;
    static constexpr size_t B_H = kL * 4;
    static constexpr size_t B_OU = 2 * kL * 4;
    static constexpr size_t B_OGX = B_OU + (size_t)kL * MB * 4;
    static constexpr size_t B_SCAN = (B_OGX + (size_t)kL * MB * 4 + 15) / 16 * 16;
    // scan block: fp32 powers P[k][MB][MB] (row-major), or for the serial scan the
    // transition as double words (hi, lo float pairs) stored column-major
    // (At[j][m] = A[m][j]), followed for MB <= 16 by its fourth power in the same form
    static constexpr size_t SCAN_F32 = (size_t)NPOW * MB * MB * 4;
    // the serial scan of MB <= 16 is blocked by four chunks and also needs Abar^4
    static constexpr bool kBlockScan = MB <= 16;
    static constexpr size_t SCAN_F64 = (size_t)MB * MB * 8 * (kBlockScan ? 2 : 1);
    __host__ __device__ static constexpr size_t scan_bytes(bool f64) { return f64 ? SCAN_F64 : SCAN_F32; }
    __host__ __device__ static constexpr size_t fwd_rec(bool f64) { return (F_SCAN + scan_bytes(f64) + 255) / 256 * 256; }
    __host__ __device__ static constexpr size_t b_coef(bool f64) { return (B_SCAN + scan_bytes(f64) + 15) / 16 * 16; }
    static constexpr size_t COEF_BYTES = ((2 * MB + 1) * 4 + 15) / 16 * 16;
    // then (orders above 4) O_L[L][MB] f32, so that a backward can recompute y from the
    // forward's chunk states with the backward record alone
    __host__ __device__ static constexpr size_t b_ol(bool f64) { return b_coef(f64) + COEF_BYTES; }
    __host__ __device__ static constexpr size_t bwd_rec(bool f64) {
        return (b_ol(f64) + (MB > 4 ? (size_t)kL * MB * 4 : 0) + 255) / 256 * 256;
    }
};

// Workspace header: a 256-byte block holding the work counter, then the records.
constexpr size_t kWsHeader = 256;

// Per-channel records: forward records at fwd_tabs, backward records at bwd_tabs
// (either may be null, not both); zeroes *counter (nullable) for the main kernel.
cudaError_t launch_chunk_setup(const float *b, const float *a, char *fwd_tabs, char *bwd_tabs,
                               unsigned long long *counter, const Batch &bt, int MB,
                               bool fp64_scan, cudaStream_t st);

}  // namespace dfilt
