// The decoupled chunked path for orders above 2 (state buckets 8..64, double-word scan).
//
// The same chunk algebra as the single-kernel path (chunk.cuh, Sec. 3.2's operator at
// chunk granularity, L = 64), split into launches so that the one serial part, the
// chunk-state scan, no longer pins a channel's tiles to one SM:
//
//   forward   E pass     E_c = R_L X_c for every chunk (FP32 FMAs on the CUDA cores,
//                        per tile, any tile on any SM), written into the chunk slots
//             scan       S_{c+1} = Abar S_c + E_c in double words; a channel is cut
//                        into spans of whole tiles scanned by different CTAs, joined
//                        by a bounded look-back (below); S_c overwrites E_c
//             Y pass     Y_c = T_g X_c + O_L S_c: T_g X_c on the tensor cores, the
//                        free response O_L S_c in FP32 on the CUDA cores
//   backward  E' pass    E'_c = (T_h^a G_c)[0:MB] (CUDA cores, like the E pass)
//             scan       S'_{c-1} = Abar' S'_c + E'_c from the end (S'_{C-1} = 0);
//                        the last state is u[0:MB] = grad_zi
//             (Y pass)   y recomputed from the forward's states when not given
//             U pass     U_c = T_h^a G_c + O^u S'_c and grad_x = T_g^a G_c + O^gx S'_c
//                        (tensor cores, free responses in FP32), u written out
//             lag sums   grad_b / grad_a lag sums per tile from u, x, y and S' (CUDA
//                        cores, exact lag blocks), one partial per tile
//             reduce     per channel, the tile partials summed in tile order (FP64)
//
// Look-back (the paper's associative operator applied to spans).  Work items are
// (channel, span) pairs handed out in order; span s > 0 first scans its own chunks
// from a zero state (its aggregate A_s), then waits (bounded) for its predecessor's
// inclusive state P_{s-1} and publishes P_s = J P_{s-1} + A_s, J = Abar^K the
// transition over K chunks of one span.  Span 0 starts from the initial state and
// publishes its end state.  A predecessor was always handed out earlier, so its CTA is
// running: no wait can deadlock.
//
// The states of span s > 0 are then S_c = S~_c + Abar^(c - c0) P_{s-1}, with S~_c the
// zero-start states of the aggregate pass.  In the forward, where the channel's
// impulse response h of 1/A decays within half a span and the table length (below
// 2^-40 of its largest value, a bound read off the impulse's chunk state norm), the
// aggregate pass writes
// S~_c to the chunk slots and keeps P_{s-1}; the Y pass computes y from S~_c, and the
// free response of the entry state, sum_m P_m h[n - m] (TDF-II state == injection at
// times m < M, Sec. 2), is added to the span's first samples afterwards in double-word
// arithmetic: one scan pass per span instead of two.  The adjoint does the same: its
// zero-start states give u and grad_x in the U pass, and hi_ufix adds the free response
// of the adjoint entry state P' (the state at the span's end in time): in reversed time
// i from the span's last sample, v[i] = sum_j h[i - j] w_j with w_j = -sum_{k>j} a_k
// P'_{k-j-1} (P' read as past outputs of the reversed all-pole recursion), extended by
// v[-1-m] = P'_m; then grad_x += sum_k b_k v[i - k] and the lag sums of v with x and y
// go into per-span partials.  Channels without a table rescan their spans from P_{s-1}.
//
// J is not formed by repeated squaring: companion-matrix powers grow transiently by
// orders of magnitude before they decay, and squaring them loses every digit (it
// diverges even in FP64 on some order-32 filters).  Instead J follows from the impulse
// response h of 1/A near n = 64K, written out in closed form (the same identities as
// the per-chunk tables, with the chunk length 64 replaced by 64K):
//     forward   J[k][m]  = -sum_{l=k+1..M} a_l h[64K + k - l - m]
//     adjoint   J'[k][m] = -sum_{j=0..M-1-m} a_{j+1+m} h[64K - 1 - k - j]
// and h near 64K comes from the impulse's state evolved over K chunks by the chunk
// transition, in double words: errors stay relative to the decayed values, as in the
// scan itself.
#pragma once

#include "chunk_pipe.cuh"

namespace dfilt {
namespace hi {

// Channel positions of one launch (the bucket's sub-list of a ragged batch, or the
// whole batch) with the prefix sums of their tiles and scan spans.
struct Plan {
    const int *list;         // bucket list (nullptr: position = channel)
    const int *list_range;   // [lo, hi) into list
    int64_t *tile_pref;      // [n + 1] tiles before each position
    int64_t *span_pref;      // [n + 1] scan spans before each position
    int *tile_pos;           // [tiles] the position of each tile
    int *span_pos;           // [spans] the position of each scan span
    int span_tiles;          // tiles per scan span (a power of two)
    int log2_span;           // log2(span_tiles)
};

__device__ __forceinline__ int64_t plan_count(const Plan &p, const Batch &bt) {
    return p.list ? (int64_t)(p.list_range[1] - p.list_range[0]) : bt.B;
}
__device__ __forceinline__ bool dbg_channel_ok(const Batch &bt, int64_t ch);
// The channel at a plan position.  Debug build: an index outside the batch records
// DFILT_ERR_BOUNDS and is replaced by channel 0, so no per-channel array is read past
// its end (the item's results are then undefined).
__device__ __forceinline__ int64_t plan_channel(const Plan &p, int64_t pos, const Batch &bt) {
    const int64_t ch = p.list ? (int64_t)p.list[p.list_range[0] + pos] : pos;
    return dbg_channel_ok(bt, ch) ? ch : 0;
}
__device__ __forceinline__ int64_t tiles_of(int64_t len) { return (len + kTileSamples - 1) / kTileSamples; }

// Debug build (-DDFILT_DEBUG): before a work item touches memory, its channel index, its
// sample range [start, start + len) and its chunk-state slot range [slot0, slot0 + nslot)
// are checked against the batch (B channels), the signal (at most bt.dbg_limit samples)
// and the slots (total / L + B + 1: one per chunk plus one spare per channel).  A failed
// check records DFILT_ERR_BOUNDS and the caller empties the item, so nothing outside the
// buffers is read or written.  The release build compiles both checks to `true`.
__device__ __forceinline__ bool dbg_channel_ok(const Batch &bt, int64_t ch) {
#ifdef DFILT_DEBUG
    const bool ok = ch >= 0 && ch < bt.B;
    if (!ok) set_status(bt.status, DFILT_ERR_BOUNDS);
    return ok;
#else
    (void)bt;
    (void)ch;
    return true;
#endif
}
__device__ __forceinline__ bool dbg_range_ok(const Batch &bt, int64_t start, int64_t len, int64_t slot0,
                                             int64_t nslot) {
#ifdef DFILT_DEBUG
    const int64_t slots = bt.total / kL + bt.B + 1;
    const bool ok = start >= 0 && len >= 0 && start + len <= bt.dbg_limit && slot0 >= 0 && nslot >= 0 &&
                    slot0 + nslot <= slots;
    if (!ok) set_status(bt.status, DFILT_ERR_BOUNDS);
    return ok;
#else
    (void)bt;
    (void)start;
    (void)len;
    (void)slot0;
    (void)nslot;
    return true;
#endif
}

// Loads without the (incoherent) L1: data another SM published in this launch.
__device__ __forceinline__ float2 ld_cg2(const float2 *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Tensor-core tile-pass modes (the E passes run on the CUDA cores, hi_epass)
enum Mode { kY = 2, kU = 3 };

// Number of lag sums per channel: grad_b[0..MB] then grad_a[1..MB]
template <int MB>
__host__ __device__ constexpr int nacc() { return 2 * MB + 1; }

}  // namespace hi

// ---- launchers (hi_tc.cu, hi_scan.cu; one translation unit per bucket) ----
// Table records: the forward record (fwd_tabs, ChunkTab<MB> layout) and the backward
// record (bwd_tabs) at the strides in bt; states: chunk slots (Mstride floats each).
struct HiArgs {
    const float *sig;       // x (forward passes, Y pass) or gy (E', U passes)
    const float *x;         // U pass: the forward's input
    const float *y;         // U pass: the forward's output
    const float *zi;        // forward scan: initial state (nullable)
    const float *acoef;     // span transitions: denominators a[B, Mstride]
    float *out;             // Y pass: y; U pass: grad_x (nullable)
    float *states;          // chunk slots: E then S (forward), E' then S' (backward)
    const float *states2;   // U pass reads S' from `states`; Y pass reads S from here
    float *gzi;             // backward scan: grad_zi (nullable)
    float *partial;         // U pass: per-tile lag sums; reduce: input
    float *gb, *ga;         // reduce outputs (nullable)
    const char *tabs;       // records used by the pass
    int64_t tab_stride;
    int tab_g, tab_ol;      // Y pass: byte offsets of g and O_L in a record
    float2 *jump;           // scan: per channel Abar^K (double words, column-major)
    float2 *jump2;          // forward's span transitions: also the adjoint's J' (nullable)
    unsigned *flags;        // scan: per item, inclusive state published
    float2 *incl;           // scan: per item inclusive state (MB double words)
    unsigned long long *counter;
    hi::Plan plan;
    int three;
    // Span entry corrections (forward): a span after a channel's first keeps the states
    // of its chunks scanned from a zero state, and its true entry state P adds the free
    // response sum_m P_m h[n - m] to y over the first samples of the span (hi_yfix).
    // Double words throughout: over long horizons the terms P_m h[n - m] cancel by many
    // orders of magnitude (the TDF-II state components of a high-order or near-unit-
    // circle filter are large and h[n - m] varies slowly in m).
    float2 *htab;           // [B][tcap] impulse response h of 1/A, h[0 .. hlen)
    int *hlen;              // [B] samples of h kept (0: the span is rescanned instead)
    int tcap;               // table length per channel (0: no corrections)
    float2 *entry;          // per span: entry state (Mstride double words; forward spans
                            // in time order, adjoint spans in processing order)
    float *span_part;       // adjoint: per span, the correction's lag sums (nacc floats)
    const float *bcoef;     // adjoint correction: numerators b[B, Nstride]
    float *ubuf;            // U pass: the zero-start adjoint u it writes (like x), read by
                            // the lag-sum kernel
};
template <int MB>
cudaError_t hi_plan(const HiArgs &h, const Batch &bt, cudaStream_t st);
template <int MB>
cudaError_t hi_jump(const HiArgs &h, const Batch &bt, bool bwd, int num_sms, cudaStream_t st);
template <int MB>
cudaError_t hi_scan(const HiArgs &h, const Batch &bt, bool bwd, int num_sms, cudaStream_t st);
template <int MB>
cudaError_t hi_tc(const HiArgs &h, const Batch &bt, int mode, int num_sms, cudaStream_t st);
template <int MB>
cudaError_t hi_reduce(const HiArgs &h, const Batch &bt, cudaStream_t st);
template <int MB>
cudaError_t hi_epass(const HiArgs &h, const Batch &bt, bool bwd, int num_sms, cudaStream_t st);
template <int MB>
cudaError_t hi_yfix(const HiArgs &h, const Batch &bt, int64_t items_bound, cudaStream_t st);
template <int MB>
cudaError_t hi_ufix(const HiArgs &h, const Batch &bt, int64_t items_bound, cudaStream_t st);
template <int MB>
cudaError_t hi_lag(const HiArgs &h, const Batch &bt, int num_sms, cudaStream_t st);

}  // namespace dfilt
