// Device helpers shared by the warp-specialised chunked kernels (forward and
// backward): tile descriptors, operand-tile addressing, named barriers, async tile
// loads, small mat-vecs, the double-word serial scan step and bounded waits.
#pragma once

#include "chunk.cuh"
#include "dword.cuh"

namespace dfilt {
namespace pipe {

constexpr uint32_t kTileBytes = kChunks * kL * 4;   // 32 KB: one signal tile
constexpr uint32_t kKBlock = kChunks * 128;         // one 32-wide K block of an operand tile
constexpr uint32_t kSmemMax = 232448;               // opt-in shared memory per block
constexpr int kNamedConv = 1, kNamedEpi = 2;
template <bool B>
struct BoolC {   // compile-time flag for generic lambdas
    static constexpr bool value = B;
};
// Warp roles shared by the warp-specialised kernels (each kernel adds its own
// converter warps): the forward's tensor-core issuer is warp 3, and both kernels'
// epilogue warps start at warp 4 (one per TMEM lane quarter, warp % 4).
constexpr int kMmaWarp = 3;
constexpr int kEpiWarp0 = 4;

struct TileDesc {
    int64_t ch;        // channel (-1: no more work)
    int64_t tstart;    // first sample (packed index)
    int64_t chunk0;    // first chunk's index in `saved`
    int32_t tlen;      // valid samples in the tile
    int32_t tab;       // table slot
    int32_t first;     // first tile of its channel (in processing order)
    int32_t M;         // channel order
    int32_t last;      // last tile of its channel (in processing order)
    int32_t seq;       // the channel's position among this CTA's channels (table slot = seq & 1)
};
static_assert(sizeof(TileDesc) == 48, "ring slots are 48 bytes");

__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

// Offset of logical 16-byte piece (row r, piece j16 of 16) in a two-K-block
// 128-byte-swizzled operand tile (row = chunk, K = sample within the chunk).
__device__ __forceinline__ uint32_t op_piece(int r, int j16) {
    return (uint32_t)((j16 >> 3) * kKBlock + r * 128 + ((((j16 & 7) ^ (r & 7))) << 4));
}

// cp.async samples [start, start+n) of src into an operand tile at `dst` (zero past n).
// Thread `t` of NT handles pieces t, t+NT, ...
template <int NT>
__device__ __forceinline__ void load_tile_async(uint32_t dst, const float *src, int64_t start,
                                                int n, bool al16, int t) {
#pragma unroll 4
    for (int q = 0; q < (2048 + NT - 1) / NT; ++q) {
        const int id = t + NT * q;
        if (id >= 2048) break;
        const int r = id >> 4, j16 = id & 15;
        const uint32_t d = dst + op_piece(r, j16);
        const int s = r * kL + j16 * 4;
        const int nv = min(max(n - s, 0), 4);
        const float *g = src + start + s;
        if (al16) {
            cp_async16(d, nv ? (const void *)g : (const void *)src, nv * 4);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                cp_async4(d + 4 * e, e < nv ? (const void *)(g + e) : (const void *)src, e < nv ? 4 : 0);
        }
    }
    cp_async_commit();
}

template <int MB>
__device__ __forceinline__ void matvec(const float *P, const float (&v)[MB], float (&out)[MB]) {
#pragma unroll
    for (int i = 0; i < MB; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < MB; ++j) acc = fmaf(P[i * MB + j], v[j], acc);
        out[i] = acc;
    }
}

// The serial chunk-state scan, s <- A s + e per chunk, in double-word arithmetic on
// the FP32 pipes (GB300's FP64 pipe is narrow; double words carry about 44 significant
// bits, far beyond what the FP32 inputs e hold).  Each product is split exactly (FMA
// TwoProduct) and its high part added with TwoSum; the low parts are summed plainly
// and folded in once per dot product.
__device__ __forceinline__ void dw_acc(float &h, float &l, float2 a, float sh, float sl) {
    const float p = a.x * sh;
    float e = fmaf(a.x, sh, -p);
    e = fmaf(a.x, sl, e);
    e = fmaf(a.y, sh, e);
    const dw s = two_sum(h, p);
    h = s.hi;
    l += s.lo + e;
}

// The scan over a tile's chunks by a group of 128 threads: TPR threads per state row
// (row r = t / TPR) each sum MB / TPR terms of the dot product, the partial double
// words are combined with shuffles (TwoSum on the high parts), and the state vector
// moves between two shared-memory buffers, one group barrier per chunk step.
//   st   : [2][MB] double words; st[0] holds the incoming state, and on return
//          st[nch & 1] holds the outgoing one
//   e    : E per chunk [nch][MB] (FP32), s_out : the state entering each chunk
//   rev  : chunks from last to first (the backward's adjoint scan)
//   sync : the group's barrier (all 128 threads call this function)
template <int MB, class Sync>
__device__ __forceinline__ void dw_scan_group(const float2 *__restrict__ At, float2 *st,
                                              const float *e, float *s_out, int nch, bool rev,
                                              int t, Sync sync) {
    constexpr int TPR = (128 / MB < MB) ? 128 / MB : MB;   // threads per row
    constexpr int JPT = MB / TPR;                          // terms per thread
    const int r = t / TPR, part = t % TPR;
    const bool active = t < MB * TPR;
    for (int k = 0; k < nch; ++k) {
        const int cc = rev ? nch - 1 - k : k;
        const float2 *cur = st + (k & 1) * MB;
        float2 *nxt = st + ((k + 1) & 1) * MB;
        float h = 0.f, l = 0.f;
        if (active) {
            if (part == 0) {
                s_out[cc * MB + r] = cur[r].x + cur[r].y;
                h = e[cc * MB + r];
            }
#pragma unroll
            for (int q = 0; q < JPT; ++q) {
                const int j = part * JPT + q;
                const float2 sj = cur[j];
                dw_acc(h, l, At[j * MB + r], sj.x, sj.y);
            }
        }
        // (every lane of the warp shuffles; rows are TPR-aligned within a warp)
#pragma unroll
        for (int off = TPR / 2; off > 0; off >>= 1) {
            const float oh = __shfl_down_sync(0xffffffffu, h, off);
            const float ol = __shfl_down_sync(0xffffffffu, l, off);
            const dw sm = two_sum(h, oh);
            h = sm.hi;
            l += ol + sm.lo;
        }
        if (active && part == 0) {
            const dw v = fast_two_sum(h, l);
            nxt[r] = make_float2(v.hi, v.lo);
        }
        sync();
    }
}

// Bounded single-thread mbarrier wait; on timeout (or a peer's abort) raise the abort
// flag and record DFILT_ERR_TIMEOUT.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, long long limit,
                                              volatile int *abort_flag, int *status) {
    for (long long it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63) {
            if (*abort_flag) return false;
            __nanosleep(32);
        }
    }
    set_status(status, DFILT_ERR_TIMEOUT);
    *abort_flag = 1;
    return false;
}

}  // namespace pipe
}  // namespace dfilt
