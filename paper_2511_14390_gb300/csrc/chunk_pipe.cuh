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

// The same scan blocked by four chunks (MB <= 16, where the serial chain's latency is
// the cost): with E'_k the chunks' inputs in processing order (zero past nch),
//   pre-pass   F_g = A^3 E'_4g + A^2 E'_4g+1 + A E'_4g+2 + E'_4g+3   (Horner, all
//              blocks at once: three group-wide steps)
//   serial     T_0 = s_in, T_{g+1} = A^4 T_g + F_g                   (nch / 4 steps)
//   post-pass  s_4g = T_g, s_4g+q = A s_4g+q-1 + E'_4g+q-1, q = 1..3  (all blocks at once)
// At4 (the fourth power) follows At in the scan block.  Scratch: vb [2][32][MB] and
// tb [33][MB] double words.  Same contract as dw_scan_group.
template <int MB, class Sync>
__device__ __forceinline__ void dw_scan_group_blocked(const float2 *__restrict__ At, float2 *st,
                                                      const float *e, float *s_out, int nch,
                                                      bool rev, int t, Sync sync, float2 *vb,
                                                      float2 *tb) {
    const float2 *__restrict__ At4 = At + MB * MB;
    const int G = (nch + 3) >> 2;
    auto chunk = [&](int k) { return rev ? nch - 1 - k : k; };   // processing order -> chunk
    auto ein = [&](int k, int r) { return k < nch ? e[chunk(k) * MB + r] : 0.f; };
    float2 *V0 = vb, *V1 = vb + 32 * MB;
    // pre-pass
    for (int it = t; it < G * MB; it += 128) V0[it] = make_float2(ein(4 * (it / MB), it % MB), 0.f);
    sync();
    for (int q = 1; q < 4; ++q) {
        const float2 *Vi = (q & 1) ? V0 : V1;
        float2 *Vo = (q & 1) ? V1 : V0;
        for (int it = t; it < G * MB; it += 128) {
            const int g = it / MB, r = it % MB;
            float h = ein(4 * g + q, r), l = 0.f;
            const float2 *v = Vi + g * MB;
#pragma unroll 4
            for (int j = 0; j < MB; ++j) dw_acc(h, l, At[j * MB + r], v[j].x, v[j].y);
            const dw o = fast_two_sum(h, l);
            Vo[it] = make_float2(o.hi, o.lo);
        }
        sync();
    }
    const float2 *F = V1;   // after the third step
    // serial pass over the blocks, TPR threads per row as in dw_scan_group
    constexpr int TPR = (128 / MB < MB) ? 128 / MB : MB;
    constexpr int JPT = MB / TPR;
    const int r = t / TPR, part = t % TPR;
    const bool active = t < MB * TPR;
    if (t < MB) tb[t] = st[t];
    sync();
    for (int g = 0; g < G; ++g) {
        const float2 *cur = tb + g * MB;
        float h = 0.f, l = 0.f;
        if (active) {
            if (part == 0) {
                h = F[g * MB + r].x;
                l = F[g * MB + r].y;
            }
#pragma unroll
            for (int q = 0; q < JPT; ++q) {
                const int j = part * JPT + q;
                const float2 sj = cur[j];
                dw_acc(h, l, At4[j * MB + r], sj.x, sj.y);
            }
        }
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
            tb[(g + 1) * MB + r] = make_float2(v.hi, v.lo);
        }
        sync();
    }
    // post-pass: the states inside each block, the outgoing one into st[nch & 1]
    float2 *out = st + (nch & 1) * MB;
    for (int it = t; it < G * MB; it += 128) {
        const int g = it / MB, rr = it % MB;
        const float2 v = tb[g * MB + rr];
        V0[it] = v;
        s_out[chunk(4 * g) * MB + rr] = v.x + v.y;
    }
    if ((nch & 3) == 0 && t < MB) out[t] = tb[G * MB + t];
    sync();
    for (int q = 1; q < 4; ++q) {
        const float2 *Vi = (q & 1) ? V0 : V1;
        float2 *Vo = (q & 1) ? V1 : V0;
        for (int it = t; it < G * MB; it += 128) {
            const int g = it / MB, rr = it % MB;
            const int k = 4 * g + q;
            float h = ein(k - 1, rr), l = 0.f;
            const float2 *v = Vi + g * MB;
#pragma unroll 4
            for (int j = 0; j < MB; ++j) dw_acc(h, l, At[j * MB + rr], v[j].x, v[j].y);
            const dw o = fast_two_sum(h, l);
            Vo[it] = make_float2(o.hi, o.lo);
            if (k < nch) s_out[chunk(k) * MB + rr] = o.hi + o.lo;
            if (k == nch) out[rr] = make_float2(o.hi, o.lo);
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
