// Internal launchers shared between the kernel translation units and the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace dfilt {

// ---- sequential algorithm (seq.cu) ----
int seq_bucket(int M);
cudaError_t launch_seq_fwd(const float *x, const float *b, const float *a, const float *zi,
                           float *y, const Batch &bt, int Mmax, cudaStream_t st);
cudaError_t launch_seq_bwd(const float *gy, const float *x, const float *y, const float *b,
                           const float *a, float *gx, float *gb, float *ga, float *gzi,
                           const Batch &bt, int Mmax, cudaStream_t st);

// ---- chunked algorithm (chunk_*.cu) ----
// Chunk length L and chunks per tensor-core tile are fixed: 64 samples x 128 chunks.
constexpr int kL = 64;
constexpr int kChunks = 128;
constexpr int kTileSamples = kL * kChunks;

// State-dimension bucket of the chunked kernels (M padded with zero coefficients).
int chunk_bucket(int M);

// High-order path choice of a call (dfilt_opts.path, .span_tiles).
struct HiOpt {
    int path = 0;         // dfilt_path
    int span_tiles = 0;   // 0 automatic
};

// Per-channel table sizes (floats / doubles) written by the setup kernels.
struct ChunkLayout {
    int MB;             // state bucket
    bool fp64_scan;     // chunk-state scan precision
    size_t fwd_tab;     // bytes of forward tables per channel
    size_t bwd_tab;     // bytes of backward tables per channel
};
ChunkLayout chunk_layout(int Mmax, int fp64_scan_opt);
// Launch plan of one call: one bucket for a fixed-shape batch, every state bucket up to
// the largest order for a ragged batch (records at the common strides).
struct ChunkPlan {
    int nb;
    ChunkLayout lay[6];
    size_t fstride, bstride;
    bool ragged;
};
// Orders 3 and 4 run in the order-8 bucket where the decoupled path may take them (it
// starts at bucket 8), so that forward, backward and the workspace sizes agree.
ChunkPlan chunk_plan(int Mmax, int fp64_opt, bool ragged, const HiOpt &ho);

// Forward-to-backward buffer (`saved`): the chunk states (channel i's chunks start at
// chunk index offsets[i] / L + i; each chunk stores Mstride floats), then, 256-byte
// aligned, the backward's per-channel tables, which the forward's setup writes so
// that the backward needs no setup of its own.
inline size_t chunk_saved_state_bytes(int64_t B, int64_t total, int Mstride) {
    return ((size_t)(total / kL + B + 1) * (size_t)Mstride * sizeof(float) + 255) / 256 * 256;
}
size_t chunk_saved_bytes(int64_t B, int64_t total, int Mmax, int fp64_opt, bool ragged,
                         const HiOpt &ho);

// Per-bucket launchers (one translation unit per bucket, compiled with -DDFILT_MB=<MB>).
template <int MB>
cudaError_t chunk_fwd_mb(const float *x, const float *zi, float *y, float *saved, const char *tabs,
                         unsigned long long *counter, const Batch &bt, bool fp64_scan, int three,
                         int num_sms, cudaStream_t st);
template <int MB>
cudaError_t chunk_bwd_mb(const float *gy, const float *x, const float *y, const float *b,
                         const float *a, const float *saved, float *gx, float *gb, float *ga,
                         float *gzi, const char *tabs, unsigned long long *counter,
                         const Batch &bt, bool fp64_scan, bool read_y, int three, int num_sms,
                         cudaStream_t st);
#define DFILT_CHUNK_BUCKETS(X) X(2) X(4) X(8) X(16) X(32) X(64)
// Largest bucket whose FP32 Hillis-Steele scan tables fit (and are used at all).
constexpr int kMaxF32ScanBucket = 16;

// Optional timing of each call's main kernel (the C ABI's kernel-timing switch): the
// launchers call it with phase 0 just before and phase 1 just after the main kernel
// (direction 0 forward, 1 backward).  A no-op while timing is off.
void timing_mark(int direction, int phase, cudaStream_t st);
// Timing classes beyond the two directions (dfilt_kernel_timing_read_classes)
enum TimingClass {
    kTimeFwd = 0, kTimeBwd = 1, kTimeScan = 2, kTimeEPass = 3, kTimeYPass = 4, kTimeUPass = 5,
    kTimeJump = 6, kTimeFused = 7
};
// Count of kernel launches issued by the library (dfilt_launch_count); every launch site
// calls it once per launch.
void note_launch();

// fp64_opt: the caller's scan option (-1 automatic per bucket, 0 off, 1 on)
cudaError_t launch_chunk_fwd(const float *x, const float *b, const float *a, const float *zi,
                             float *y, float *saved, void *ws, const Batch &bt, int Mmax,
                             int fp64_opt, int precision, int num_sms, cudaStream_t st,
                             const HiOpt &ho);
cudaError_t launch_chunk_bwd(const float *gy, const float *x, const float *y, const float *b,
                             const float *a, const float *saved, float *gx, float *gb,
                             float *ga, float *gzi, void *ws, const Batch &bt, int Mmax,
                             int fp64_opt, int precision, int num_sms, cudaStream_t st,
                             const HiOpt &ho);
// Workspace bytes; `total` = samples of the batch (the decoupled path's per-span and
// per-tile records grow with it).
size_t chunk_fwd_ws_bytes(int64_t B, int64_t total, int Mmax, int fp64_opt, bool ragged,
                          const HiOpt &ho);
size_t chunk_bwd_ws_bytes(int64_t B, int64_t total, int Mmax, int fp64_opt, bool ragged,
                          const HiOpt &ho);
// Span length (tiles) the decoupled path uses for a bucket of a call.
int hi_span_tiles(int MB, int64_t B, int64_t total, bool ragged, int num_sms, const HiOpt &ho);
// Tuning table of the decoupled scan per state bucket (0 = automatic); the scan's
// default chains (CTAs) per SM.
bool hi_tuning_set(int MB, int span_tiles, int chains_per_sm);
void hi_tuning_get(int MB, int *span_tiles, int *chains_per_sm);
constexpr int hi_scan_chains_default(int MB) { return MB <= 16 ? 16 : (MB == 32 ? 8 : 4); }

// Tensor map of a signal viewed as rows of one chunk (L floats), 3-D so that one box
// {32 floats, 1 half, 128 rows} is one 128-byte-swizzled K block of a tensor-core
// operand tile.  Returns false when the layout does not allow it (rows not aligned to
// chunk boundaries, misaligned base) -- callers then use plain async copies.
bool make_chunk_tmap(CUtensorMap *map, const float *base, int64_t total);

}  // namespace dfilt
