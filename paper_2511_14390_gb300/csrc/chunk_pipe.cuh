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

// One step of the serial chunk-state scan, s <- A s + e, in double-word arithmetic on
// the FP32 pipes (GB300's FP64 pipe is narrow; double words carry about 44 significant
// bits, far beyond what the FP32 inputs e hold).  One warp: lane r < MB holds state
// component r in sa and (MB = 64) component r + 32 in sb.  At is the transition stored
// column-major as (hi, lo) pairs, At[j * MB + m] = A[m][j].  Each product is split
// exactly (FMA TwoProduct) and its high part added with TwoSum; the low parts are
// summed plainly and folded in once at the end.
__device__ __forceinline__ void dw_acc(float &h, float &l, float2 a, float sh, float sl) {
    const float p = a.x * sh;
    float e = fmaf(a.x, sh, -p);
    e = fmaf(a.x, sl, e);
    e = fmaf(a.y, sh, e);
    const dw s = two_sum(h, p);
    h = s.hi;
    l += s.lo + e;
}
template <int MB>
__device__ __forceinline__ void dw_scan_step(const float2 *__restrict__ At, float ea, float eb,
                                             dw &sa, dw &sb, int lane) {
    float ah = ea, al = 0.f, bh = eb, bl = 0.f;
#pragma unroll 8
    for (int j = 0; j < MB; ++j) {
        const float sh = __shfl_sync(0xffffffffu, j < 32 ? sa.hi : sb.hi, j & 31);
        const float sl = __shfl_sync(0xffffffffu, j < 32 ? sa.lo : sb.lo, j & 31);
        if (lane < MB) dw_acc(ah, al, At[j * MB + lane], sh, sl);
        if (lane + 32 < MB) dw_acc(bh, bl, At[j * MB + lane + 32], sh, sl);
    }
    sa = fast_two_sum(ah, al);
    sb = fast_two_sum(bh, bl);
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
