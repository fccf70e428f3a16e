// Host-side dispatch of the chunked algorithm: state-dimension bucket, scan precision,
// workspace sizes, and the setup + main kernel launches per bucket.
#include <cudaTypedefs.h>
#include <mutex>
#include <type_traits>

#include "chunk.cuh"
#include "hi.cuh"

namespace dfilt {

#define DFILT_HI_BUCKETS(X) X(8) X(16) X(32) X(64)
#define DFILT_HI_EXTERN(V)                                                                        \
    extern template cudaError_t hi_plan<V>(const HiArgs &, const Batch &, cudaStream_t);          \
    extern template cudaError_t hi_jump<V>(const HiArgs &, const Batch &, bool, int, cudaStream_t); \
    extern template cudaError_t hi_scan<V>(const HiArgs &, const Batch &, bool, int, cudaStream_t); \
    extern template cudaError_t hi_tc<V>(const HiArgs &, const Batch &, int, int, cudaStream_t);   \
    extern template cudaError_t hi_reduce<V>(const HiArgs &, const Batch &, cudaStream_t);        \
    extern template cudaError_t hi_epass<V>(const HiArgs &, const Batch &, bool, int, cudaStream_t); \
    extern template cudaError_t hi_yfix<V>(const HiArgs &, const Batch &, int64_t, cudaStream_t);    \
    extern template cudaError_t hi_ufix<V>(const HiArgs &, const Batch &, int64_t, cudaStream_t);    \
    extern template cudaError_t hi_lag<V>(const HiArgs &, const Batch &, int, cudaStream_t);
DFILT_HI_BUCKETS(DFILT_HI_EXTERN)
#undef DFILT_HI_EXTERN

#define DFILT_EXTERN(V)                                                                          \
    extern template cudaError_t chunk_fwd_mb<V>(const float *, const float *, float *, float *, \
                                                const char *, unsigned long long *, const Batch &, \
                                                bool, int, int, cudaStream_t);                   \
    extern template cudaError_t chunk_bwd_mb<V>(                                                 \
        const float *, const float *, const float *, const float *, const float *,              \
        const float *, float *, float *, float *, float *, const char *, unsigned long long *,  \
        const Batch &, bool, bool, int, int, cudaStream_t);
DFILT_CHUNK_BUCKETS(DFILT_EXTERN)
#undef DFILT_EXTERN

bool make_chunk_tmap(CUtensorMap *map, const float *base, int64_t total) {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!encode || !base || total <= 0 || total % kL != 0) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    const cuuint64_t rows = (cuuint64_t)(total / kL);
    if (rows > 0xFFFFFFFFull) return false;
    const cuuint64_t dims[3] = {32, 2, rows};
    const cuuint64_t strides[2] = {128, kL * 4};
    const cuuint32_t box[3] = {32, 1, (cuuint32_t)kChunks};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base),
                              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int chunk_bucket(int M) {
    for (int mb : {2, 4, 8, 16, 32, 64})
        if (M <= mb) return mb;
    return -1;
}

ChunkLayout chunk_layout(int Mmax, int fp64_scan_opt) {
    ChunkLayout l;
    l.MB = chunk_bucket(Mmax);
    // FP32 powers of the chunk transition stay accurate for orders <= 2 up to pole radius
    // 0.9995; from order 3 on, the transient growth of companion-matrix powers costs an
    // FP32 scan accuracy (measured 21x the double-word scan's error at order 4, radius
    // 0.99-0.9995) and diverges on some high-order filters, so the automatic choice
    // there is the serial scan in double words (FP64-class accuracy; the only one above
    // the FP32 table bucket limit).
    l.fp64_scan = fp64_scan_opt < 0 ? (Mmax > 2) : (fp64_scan_opt != 0);
    if (l.MB > kMaxF32ScanBucket) l.fp64_scan = true;
    size_t f = 0, b = 0;
    switch (l.MB) {
#define X(V)                                   \
    case V:                                    \
        f = ChunkTab<V>::fwd_rec(l.fp64_scan); \
        b = ChunkTab<V>::bwd_rec(l.fp64_scan); \
        break;
        DFILT_CHUNK_BUCKETS(X)
#undef X
    }
    l.fwd_tab = f;
    l.bwd_tab = b;
    return l;
}

// the decoupled path's state buckets (8 holds orders 3..8 when the path may be taken)
static bool hi_path_allowed(const HiOpt &ho) { return ho.path != DFILT_PATH_FUSED; }

// Per-bucket plan: a fixed-shape batch is one bucket; a ragged batch runs every state
// bucket up to its largest order as its own launch pair (setup + main kernel) over the
// channels of that bucket, with records at a common stride.  Where the decoupled path may
// run, the double-word-scan orders 3 and 4 join bucket 8.
ChunkPlan chunk_plan(int Mmax, int fp64_opt, bool ragged, const HiOpt &ho) {
    ChunkPlan p{};
    p.ragged = ragged;
    auto lay_of = [&](int m) {
        ChunkLayout l = chunk_layout(m, fp64_opt);
        if (l.MB == 4 && l.fp64_scan && hi_path_allowed(ho)) l = chunk_layout(8, fp64_opt);
        return l;
    };
    if (!ragged) {
        p.nb = 1;
        p.lay[0] = lay_of(Mmax);
    } else {
        const int top = chunk_bucket(Mmax);
        p.nb = 0;
        for (int mb : {2, 4, 8, 16, 32, 64}) {
            if (mb > top) break;
            const ChunkLayout l = lay_of(mb);
            if (p.nb > 0 && p.lay[p.nb - 1].MB == l.MB) continue;   // merged into the next
            p.lay[p.nb++] = l;
        }
        if (p.nb > 0 && p.lay[p.nb - 1].MB < top) p.lay[p.nb++] = lay_of(top);
    }
    for (int j = 0; j < p.nb; ++j) {
        p.fstride = p.lay[j].fwd_tab > p.fstride ? p.lay[j].fwd_tab : p.fstride;
        p.bstride = p.lay[j].bwd_tab > p.bstride ? p.lay[j].bwd_tab : p.bstride;
    }
    return p;
}

// channel list of a ragged batch: B bucket-sorted channel indices, then nb+1 bucket starts
static size_t list_bytes(int64_t B, bool ragged) {
    return ragged ? ((size_t)(B + 16) * sizeof(int) + 255) / 256 * 256 : 0;
}

// ---------------------------------------------------------------------------
// Decoupled high-order path: which buckets take it, and its workspace blocks
// ---------------------------------------------------------------------------
static bool hi_eligible(const ChunkLayout &l, const HiOpt &ho) {
    return l.MB >= 8 && l.fp64_scan && ho.path != DFILT_PATH_FUSED;
}

// Blocks of the decoupled path behind the fused path's workspace (all 256-byte aligned):
//   ctl      work counters (4 per bucket)
//   pref     per hi bucket: tile and span prefix sums over its channel positions
//   pos      per hi bucket: the channel position of every tile and every scan span
//   jump     per channel: the span transition (MB x MB double words)
//   flags    per scan item: inclusive state published;  incl: that state
//   (backward) sprime: the adjoint's chunk states; ybuf: y recomputed; partial: lag
//   sums per tile
struct HiWs {
    size_t ctl = 0, pref = 0, pos = 0, jump = 0, flags = 0, incl = 0, sprime = 0, ybuf = 0, partial = 0;
    size_t entry_b = 0, span_part = 0;   // backward: adjoint span entry states, their lag sums
    size_t ubuf = 0;                     // backward: the U pass's adjoint u (total floats)
    size_t end = 0;
    size_t ctl_bytes = 0;   // the block cleared once per call (counters)
    int nhi = 0, mbmax = 0;
    int64_t items_bound = 0;
};
static size_t al256(size_t v) { return (v + 255) / 256 * 256; }

static HiWs hi_ws(size_t base, const ChunkPlan &p, int64_t B, int64_t total, int Mstride,
                  bool bwd, const HiOpt &ho) {
    HiWs h;
    for (int j = 0; j < p.nb; ++j)
        if (hi_eligible(p.lay[j], ho)) {
            ++h.nhi;
            h.mbmax = p.lay[j].MB > h.mbmax ? p.lay[j].MB : h.mbmax;
        }
    h.end = base;
    if (!h.nhi) return h;
    // every span holds at least one tile and every channel ends at most one partial
    // tile: items and tiles per bucket are at most total / 8192 + B + 1
    h.items_bound = total / kTileSamples + B + 1;
    size_t o = al256(base);
    h.ctl = o;
    h.ctl_bytes = al256((size_t)h.nhi * 8 * sizeof(unsigned long long));   // 8 per bucket
    o += h.ctl_bytes;
    h.pref = o;
    o += al256((size_t)h.nhi * 2 * (B + 1) * sizeof(int64_t));
    h.pos = o;
    o += al256((size_t)h.nhi * 2 * h.items_bound * sizeof(int));
    h.jump = o;
    o += al256((size_t)B * h.mbmax * h.mbmax * 8);
    h.flags = o;
    o += al256((size_t)h.items_bound * 4);
    h.incl = o;
    o += al256((size_t)h.items_bound * h.mbmax * 8);
    if (bwd) {
        h.sprime = o;
        o += chunk_saved_state_bytes(B, total, Mstride);
        h.ybuf = o;
        o += al256((size_t)total * 4);
        h.partial = o;
        o += al256((size_t)h.items_bound * (2 * h.mbmax + 1) * 4);
        h.entry_b = o;
        o += al256((size_t)h.items_bound * Mstride * 8);
        h.span_part = o;
        o += al256((size_t)h.items_bound * (2 * h.mbmax + 1) * 4);
        h.ubuf = o;
        o += al256((size_t)total * 4);
    }
    h.end = o;
    return h;
}

static size_t fused_fwd_ws(int64_t B, const ChunkPlan &p, bool ragged) {
    return kWsHeader + (size_t)B * p.fstride + list_bytes(B, ragged);
}
static size_t fused_bwd_ws(int64_t B, const ChunkPlan &p, bool ragged) {
    return kWsHeader + (size_t)B * p.bstride + list_bytes(B, ragged);
}

size_t chunk_fwd_ws_bytes(int64_t B, int64_t total, int Mmax, int fp64_opt, bool ragged,
                          const HiOpt &ho) {
    const ChunkPlan p = chunk_plan(Mmax, fp64_opt, ragged, ho);
    return hi_ws(fused_fwd_ws(B, p, ragged), p, B, total, Mmax, false, ho).end;
}

size_t chunk_bwd_ws_bytes(int64_t B, int64_t total, int Mmax, int fp64_opt, bool ragged,
                          const HiOpt &ho) {
    const ChunkPlan p = chunk_plan(Mmax, fp64_opt, ragged, ho);
    return hi_ws(fused_bwd_ws(B, p, ragged), p, B, total, Mmax, true, ho).end;
}

// ---------------------------------------------------------------------------
// Tuning table of the decoupled scan, per state bucket: span length (tiles) and chains
// per SM; 0 = the rule below.  Set by dfilt_tuning_set (the package's tuner measures
// candidates and installs the best).
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
int g_tune_span[7] = {};     // index log2(MB) - 1 (MB = 2..64)
int g_tune_chains[7] = {};
int tune_index(int MB) {
    int i = 0;
    while ((2 << i) < MB && i < 6) ++i;
    return i;
}
}  // namespace

bool hi_tuning_set(int MB, int span_tiles, int chains_per_sm) {
    if (chunk_bucket(MB) != MB || span_tiles < 0 || span_tiles > 4096 ||
        (span_tiles & (span_tiles - 1)) != 0 || chains_per_sm < 0 || chains_per_sm > 32)
        return false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_span[tune_index(MB)] = span_tiles;
    g_tune_chains[tune_index(MB)] = chains_per_sm;
    return true;
}
void hi_tuning_get(int MB, int *span_tiles, int *chains_per_sm) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (span_tiles) *span_tiles = g_tune_span[tune_index(MB)];
    if (chains_per_sm) *chains_per_sm = g_tune_chains[tune_index(MB)];
}

// Span length of the decoupled scan (tiles, a power of two): the caller's choice, else
// the tuning table's, else about half of the tiles per chain (rounded down to a power of
// two), measured best on the order-16, orders-64 and ragged workloads: shorter spans
// add rescans (every span after a channel's first scans twice), longer ones lengthen the
// longest chain.
int hi_span_tiles(int MB, int64_t B, int64_t total, bool ragged, int num_sms, const HiOpt &ho) {
    if (ho.span_tiles > 0) return ho.span_tiles;
    int st_tab = 0, ch_tab = 0;
    hi_tuning_get(MB, &st_tab, &ch_tab);
    if (st_tab > 0) return st_tab;
    const int64_t chains = (int64_t)num_sms * (ch_tab > 0 ? ch_tab : hi_scan_chains_default(MB));
    int64_t tiles;
    if (!ragged) {
        const int64_t T = B > 0 ? total / B : 0;
        tiles = B * ((T + kTileSamples - 1) / kTileSamples);
    } else {
        tiles = total / kTileSamples + B;
    }
    const int64_t want = tiles / (2 * chains);
    int st = 1;
    while (2 * st <= want && st < 4096) st <<= 1;
    return st;
}

// `saved` = chunk states | backward records | (decoupled path) the adjoint's span
// transitions J' per channel, formed by the forward together with its own
static size_t saved_jump_off(int64_t B, int64_t total, int Mmax, const ChunkPlan &p) {
    return al256(chunk_saved_state_bytes(B, total, Mmax) + (size_t)B * p.bstride);
}

// Table length of the forward's span entry corrections (samples of h per channel, one
// double word each): a power of two from 4096 to 65536, at most an eighth of the mean
// channel length, so the tables add at most 1 byte per sample of the batch to `saved`
// (beyond that floor).  A channel whose impulse response does not decay within its span
// and the table has its spans rescanned.
static int hi_tcap(int64_t B, int64_t total) {
    const int64_t per = B > 0 ? total / (8 * B) : 0;
    int64_t t = 4096;
    while (t * 2 <= per && t < 65536) t *= 2;
    return (int)t;
}

// The decoupled path's part of `saved`, behind the chunk states and backward records:
//   jump2   per channel: the adjoint's span transition J' (formed by the forward)
//   htab    per channel: h of 1/A over the correction region (tcap floats)
//   hlen    per channel: samples of h kept (0: no correction)
//   entry   per hi bucket and span: the forward's span entry state (Mstride floats)
struct HiSaved {
    size_t jump2 = 0, htab = 0, hlen = 0, entry = 0, end = 0;
    int tcap = 0;
};
static HiSaved hi_saved(int64_t B, int64_t total, int Mmax, const ChunkPlan &p, const HiWs &hw) {
    HiSaved sv;
    sv.jump2 = saved_jump_off(B, total, Mmax, p);
    size_t o = sv.jump2;
    if (hw.nhi) {
        o += al256((size_t)B * hw.mbmax * hw.mbmax * 8);
        sv.tcap = hi_tcap(B, total);
        sv.htab = o;
        o += al256((size_t)B * sv.tcap * 8);
        sv.hlen = o;
        o += al256((size_t)B * 4);
        sv.entry = o;
        o += al256((size_t)hw.nhi * hw.items_bound * Mmax * 8);
    }
    sv.end = o;
    return sv;
}

size_t chunk_saved_bytes(int64_t B, int64_t total, int Mmax, int fp64_opt, bool ragged,
                         const HiOpt &ho) {
    const ChunkPlan p = chunk_plan(Mmax, fp64_opt, ragged, ho);
    const HiWs hw = hi_ws(0, p, B, total, Mmax, false, ho);
    return hi_saved(B, total, Mmax, p, hw).end;
}

// Point a bucket's call at the correction blocks of `saved` (bucket rank hj).
static void hi_saved_ptrs(HiArgs &a, char *saved, const HiSaved &sv, const HiWs &hw, int hj,
                          int Mmax) {
    a.htab = reinterpret_cast<float2 *>(saved + sv.htab);
    a.hlen = reinterpret_cast<int *>(saved + sv.hlen);
    a.tcap = sv.tcap;
    a.entry = reinterpret_cast<float2 *>(saved + sv.entry) + (size_t)hj * hw.items_bound * Mmax;
}

namespace {

// Sort the channels of a ragged batch by state bucket (one block; order within a bucket
// is arbitrary, which no result depends on): list[starts[j] .. starts[j+1]) are the
// channels of bucket j (orders up to be.mb[j]; the last bucket takes the rest).
struct BucketEdges {
    int mb[8];   // bucket j takes the orders above mb[j-1] up to mb[j]
};

__global__ void __launch_bounds__(1024) bucket_channels_kernel(const int *__restrict__ Ms, int64_t B,
                                                               int Mstride, int nb, BucketEdges be,
                                                               int *__restrict__ list,
                                                               int *__restrict__ starts) {
    __shared__ int cnt[8], pos[8];
    if (threadIdx.x < 8) cnt[threadIdx.x] = 0;
    __syncthreads();
    auto bucket = [&](int64_t i) {
        int m = Ms[i];
        m = m < 1 ? 1 : (m > Mstride ? Mstride : m);
        int j = 0;
        while (j < nb - 1 && m > be.mb[j]) ++j;
        return j;
    };
    for (int64_t i = threadIdx.x; i < B; i += blockDim.x) atomicAdd(&cnt[bucket(i)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int j = 0; j <= nb; ++j) {
            starts[j] = acc;
            if (j < nb) {
                pos[j] = acc;
                acc += cnt[j];
            }
        }
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < B; i += blockDim.x) list[atomicAdd(&pos[bucket(i)], 1)] = (int)i;
}

BucketEdges edges(const ChunkPlan &p) {
    BucketEdges be{};
    for (int j = 0; j < p.nb; ++j) be.mb[j] = p.lay[j].MB;
    return be;
}

}  // namespace

// The decoupled path for bucket j of a call (forward or backward), launched on `st`.
struct HiCall {
    HiArgs a;
    Batch bt;
    int MB;
};

template <class F>
static cudaError_t hi_switch(int MB, F f) {
    switch (MB) {
        case 8: return f(std::integral_constant<int, 8>{});
        case 16: return f(std::integral_constant<int, 16>{});
        case 32: return f(std::integral_constant<int, 32>{});
        case 64: return f(std::integral_constant<int, 64>{});
        default: return cudaErrorInvalidValue;
    }
}

// Fill the plan pointers of bucket `hj` (its rank among the call's hi buckets).
static void hi_plan_ptrs(HiArgs &a, char *w, const HiWs &hw, int hj, int64_t B, int span_tiles) {
    int64_t *pref = reinterpret_cast<int64_t *>(w + hw.pref) + (size_t)hj * 2 * (B + 1);
    a.plan.tile_pref = pref;
    a.plan.span_pref = pref + (B + 1);
    int *pos = reinterpret_cast<int *>(w + hw.pos) + (size_t)hj * 2 * hw.items_bound;
    a.plan.tile_pos = pos;
    a.plan.span_pos = pos + hw.items_bound;
    a.plan.span_tiles = span_tiles;
    int lg = 0;
    while ((1 << lg) < span_tiles) ++lg;
    a.plan.log2_span = lg;
    a.jump = reinterpret_cast<float2 *>(w + hw.jump);
    a.flags = reinterpret_cast<unsigned *>(w + hw.flags);
    a.incl = reinterpret_cast<float2 *>(w + hw.incl);
}

cudaError_t launch_chunk_fwd(const float *x, const float *b, const float *a, const float *zi,
                             float *y, float *saved, void *ws, const Batch &bt, int Mmax,
                             int fp64_opt, int precision, int num_sms, cudaStream_t st,
                             const HiOpt &ho) {
    const bool ragged = bt.offsets != nullptr && bt.Ms != nullptr;
    const ChunkPlan p = chunk_plan(Mmax, fp64_opt, ragged, ho);
    char *w = static_cast<char *>(ws);
    auto *counters = reinterpret_cast<unsigned long long *>(w);   // one per bucket
    // with a saved buffer, the same setup launch also writes the backward's tables into it
    char *btabs = saved ? reinterpret_cast<char *>(saved) + chunk_saved_state_bytes(bt.B, bt.total, Mmax)
                        : nullptr;
    const HiWs hw = hi_ws(fused_fwd_ws(bt.B, p, ragged), p, bt.B, bt.total, Mmax, false, ho);
    Batch bb[8];
    int *list = reinterpret_cast<int *>(w + kWsHeader + (size_t)bt.B * p.fstride);
    if (ragged) {
        bucket_channels_kernel<<<1, 1024, 0, st>>>(bt.Ms, bt.B, bt.Mstride, p.nb, edges(p), list,
                                                   list + bt.B); note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // the decoupled path needs `saved` for its chunk states
    bool use_hi[8] = {};
    bool any_hi = false;
    for (int j = 0; j < p.nb; ++j) {
        use_hi[j] = saved != nullptr && hw.nhi > 0 && hi_eligible(p.lay[j], ho);
        any_hi |= use_hi[j];
    }
    if (any_hi) {
        const cudaError_t e = cudaMemsetAsync(w + hw.ctl, 0, hw.ctl_bytes, st);
        if (e != cudaSuccess) return e;
    }
    for (int j = 0; j < p.nb; ++j) {
        bb[j] = bt;
        if (ragged) {
            bb[j].list = list;
            bb[j].list_range = list + bt.B + j;
            bb[j].fwd_stride = (int64_t)p.fstride;
            bb[j].bwd_stride = (int64_t)p.bstride;
        }
        const cudaError_t e = launch_chunk_setup(b, a, w + kWsHeader, btabs, counters + j, bb[j],
                                                 p.lay[j].MB, p.lay[j].fp64_scan, st);
        if (e != cudaSuccess) return e;
    }
    const int three = precision == DFILT_PREC_TF32X3 ? 1 : 0;
    cudaError_t e = cudaSuccess;
    timing_mark(0, 0, st);
    int hj = 0;
    for (int j = 0; j < p.nb && e == cudaSuccess; ++j) {
        if (use_hi[j]) {
            const int MB = p.lay[j].MB;
            HiArgs h{};
            h.sig = x;
            h.zi = zi;
            h.acoef = a;
            h.out = y;
            h.states = saved;
            h.states2 = saved;
            h.tabs = w + kWsHeader;
            h.tab_stride = ragged ? (int64_t)p.fstride : (int64_t)p.lay[j].fwd_tab;
            h.three = three;
            h.plan.list = bb[j].list;
            h.plan.list_range = bb[j].list_range;
            const int stl = hi_span_tiles(MB, bt.B, bt.total, ragged, num_sms, ho);
            hi_plan_ptrs(h, w, hw, hj, bt.B, stl);
            const HiSaved sv = hi_saved(bt.B, bt.total, Mmax, p, hw);
            hi_saved_ptrs(h, reinterpret_cast<char *>(saved), sv, hw, hj, Mmax);
            auto *ctl = reinterpret_cast<unsigned long long *>(w + hw.ctl) + 8 * hj;
            ++hj;
            e = hi_switch(MB, [&](auto mbc) -> cudaError_t {
                constexpr int V = decltype(mbc)::value;
                using Tab = ChunkTab<V>;
                HiArgs q = h;
                cudaError_t r = hi_plan<V>(q, bb[j], st);
                if (r != cudaSuccess) return r;
                q.counter = ctl + 0;
                timing_mark(kTimeEPass, 0, st);
                r = hi_epass<V>(q, bb[j], false, num_sms, st);   // E_c into the slots
                timing_mark(kTimeEPass, 1, st);
                if (r != cudaSuccess) return r;
                q.jump2 = reinterpret_cast<float2 *>(reinterpret_cast<char *>(saved) + sv.jump2);
                timing_mark(kTimeJump, 0, st);
                r = hi_jump<V>(q, bb[j], false, num_sms, st);   // J, and J' for the backward
                timing_mark(kTimeJump, 1, st);
                if (r != cudaSuccess) return r;
                r = cudaMemsetAsync(q.flags, 0, (size_t)hw.items_bound * 4, st);
                if (r != cudaSuccess) return r;
                q.counter = ctl + 1;
                timing_mark(kTimeScan, 0, st);
                r = hi_scan<V>(q, bb[j], false, num_sms, st);   // S_c over the slots
                timing_mark(kTimeScan, 1, st);
                if (r != cudaSuccess) return r;
                q.counter = ctl + 2;
                q.tab_g = (int)Tab::F_G;
                q.tab_ol = (int)Tab::F_OL;
                timing_mark(kTimeYPass, 0, st);
                r = hi_tc<V>(q, bb[j], hi::kY, num_sms, st);   // y
                if (r == cudaSuccess) r = hi_yfix<V>(q, bb[j], hw.items_bound, st);   // span entries
                timing_mark(kTimeYPass, 1, st);
                return r;
            });
            continue;
        }
        timing_mark(kTimeFused, 0, st);
        switch (p.lay[j].MB) {
#define X(V)                                                                                   \
    case V:                                                                                    \
        e = chunk_fwd_mb<V>(x, zi, y, saved, w + kWsHeader, counters + j, bb[j],               \
                            p.lay[j].fp64_scan, three, num_sms, st);                           \
        break;
            DFILT_CHUNK_BUCKETS(X)
#undef X
            default: e = cudaErrorInvalidValue;
        }
        timing_mark(kTimeFused, 1, st);
    }
    timing_mark(0, 1, st);
    return e;
}

cudaError_t launch_chunk_bwd(const float *gy, const float *x, const float *y, const float *b,
                             const float *a, const float *saved, float *gx, float *gb, float *ga,
                             float *gzi, void *ws, const Batch &bt, int Mmax, int fp64_opt,
                             int precision, int num_sms, cudaStream_t st, const HiOpt &ho) {
    const bool ragged = bt.offsets != nullptr && bt.Ms != nullptr;
    const ChunkPlan p = chunk_plan(Mmax, fp64_opt, ragged, ho);
    const bool read_y = saved == nullptr;   // y is recomputed whenever the chunk states exist
    if (read_y && (!y || chunk_bucket(Mmax) > 32)) return cudaErrorNotSupported;
    char *wsc = static_cast<char *>(ws);
    auto *counters = reinterpret_cast<unsigned long long *>(wsc);   // one per bucket
    // the forward's setup left the backward tables behind the chunk states
    const char *tabs = saved ? reinterpret_cast<const char *>(saved) +
                                   chunk_saved_state_bytes(bt.B, bt.total, Mmax)
                             : wsc + kWsHeader;
    const HiWs hw = hi_ws(fused_bwd_ws(bt.B, p, ragged), p, bt.B, bt.total, Mmax, true, ho);
    Batch bb[8];
    int *list = reinterpret_cast<int *>(wsc + kWsHeader + (size_t)bt.B * p.bstride);
    cudaError_t e = cudaSuccess;
    if (ragged) {
        bucket_channels_kernel<<<1, 1024, 0, st>>>(bt.Ms, bt.B, bt.Mstride, p.nb, edges(p), list,
                                                   list + bt.B); note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    bool use_hi[8] = {};
    bool any_hi = false;
    for (int j = 0; j < p.nb; ++j) {
        use_hi[j] = saved != nullptr && hw.nhi > 0 && hi_eligible(p.lay[j], ho);
        any_hi |= use_hi[j];
    }
    if (saved) e = cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * p.nb, st);
    if (e != cudaSuccess) return e;
    if (any_hi) e = cudaMemsetAsync(wsc + hw.ctl, 0, hw.ctl_bytes, st);
    if (e != cudaSuccess) return e;
    for (int j = 0; j < p.nb; ++j) {
        bb[j] = bt;
        if (ragged) {
            bb[j].list = list;
            bb[j].list_range = list + bt.B + j;
            bb[j].fwd_stride = (int64_t)p.fstride;
            bb[j].bwd_stride = (int64_t)p.bstride;
        }
        if (!saved) {
            e = launch_chunk_setup(b, a, nullptr, wsc + kWsHeader, counters + j, bb[j], p.lay[j].MB,
                                   p.lay[j].fp64_scan, st);
            if (e != cudaSuccess) return e;
        }
    }
    const int three = precision == DFILT_PREC_TF32X3 ? 1 : 0;
    timing_mark(1, 0, st);
    int hj = 0;
    for (int j = 0; j < p.nb && e == cudaSuccess; ++j) {
        if (use_hi[j]) {
            const int MB = p.lay[j].MB;
            HiArgs h{};
            h.acoef = a;
            h.tabs = tabs;
            h.tab_stride = ragged ? (int64_t)p.bstride : (int64_t)p.lay[j].bwd_tab;
            h.three = three;
            h.plan.list = bb[j].list;
            h.plan.list_range = bb[j].list_range;
            const int stl = hi_span_tiles(MB, bt.B, bt.total, ragged, num_sms, ho);
            hi_plan_ptrs(h, wsc, hw, hj, bt.B, stl);
            auto *ctl = reinterpret_cast<unsigned long long *>(wsc + hw.ctl) + 8 * hj;
            ++hj;
            float *sprime = reinterpret_cast<float *>(wsc + hw.sprime);
            float *ybuf = reinterpret_cast<float *>(wsc + hw.ybuf);
            h.partial = reinterpret_cast<float *>(wsc + hw.partial);
            const HiSaved sv = hi_saved(bt.B, bt.total, Mmax, p, hw);
            const int hj_this = hj - 1;
            // the forward's correction table; this call's own span entry states
            hi_saved_ptrs(h, const_cast<char *>(reinterpret_cast<const char *>(saved)), sv, hw, hj_this, Mmax);
            h.entry = reinterpret_cast<float2 *>(wsc + hw.entry_b);
            h.span_part = reinterpret_cast<float *>(wsc + hw.span_part);
            h.bcoef = b;
            h.ubuf = reinterpret_cast<float *>(wsc + hw.ubuf);
            e = hi_switch(MB, [&](auto mbc) -> cudaError_t {
                constexpr int V = decltype(mbc)::value;
                using Tab = ChunkTab<V>;
                HiArgs q = h;
                cudaError_t r = hi_plan<V>(q, bb[j], st);
                if (r != cudaSuccess) return r;
                // E'_c = (T_h^a G_c)[0:MB] into the adjoint's slots
                q.sig = gy;
                q.states = sprime;
                q.counter = ctl + 0;
                timing_mark(kTimeEPass, 0, st);
                r = hi_epass<V>(q, bb[j], true, num_sms, st);
                timing_mark(kTimeEPass, 1, st);
                if (r != cudaSuccess) return r;
                // the adjoint's span transitions, formed by the forward
                q.jump = reinterpret_cast<float2 *>(const_cast<char *>(reinterpret_cast<const char *>(saved)) +
                                                    sv.jump2);
                r = cudaMemsetAsync(q.flags, 0, (size_t)hw.items_bound * 4, st);
                if (r != cudaSuccess) return r;
                q.counter = ctl + 1;
                q.gzi = gzi;
                timing_mark(kTimeScan, 0, st);
                r = hi_scan<V>(q, bb[j], true, num_sms, st);   // S'_c, grad_zi
                timing_mark(kTimeScan, 1, st);
                if (r != cudaSuccess) return r;
                const float *yv = y;
                if (!yv) {
                    // y recomputed from the forward's chunk states (Y pass, backward record)
                    HiArgs qy = q;
                    qy.sig = x;
                    qy.states2 = saved;
                    qy.out = ybuf;
                    qy.counter = ctl + 2;
                    qy.tab_g = (int)Tab::B_G;
                    qy.tab_ol = (int)Tab::b_ol(true);
                    hi_saved_ptrs(qy, const_cast<char *>(reinterpret_cast<const char *>(saved)), sv, hw,
                                  hj_this, Mmax);
                    timing_mark(kTimeYPass, 0, st);
                    r = hi_tc<V>(qy, bb[j], hi::kY, num_sms, st);
                    if (r == cudaSuccess) r = hi_yfix<V>(qy, bb[j], hw.items_bound, st);
                    timing_mark(kTimeYPass, 1, st);
                    if (r != cudaSuccess) return r;
                    yv = ybuf;
                }
                q.sig = gy;
                q.x = x;
                q.y = yv;
                q.out = gx;
                q.counter = ctl + 3;
                timing_mark(kTimeUPass, 0, st);
                r = hi_tc<V>(q, bb[j], hi::kU, num_sms, st);   // grad_x, u
                if (r != cudaSuccess) return r;
                q.counter = ctl + 4;
                r = hi_lag<V>(q, bb[j], num_sms, st);   // lag sums per tile
                if (r != cudaSuccess) return r;
                r = hi_ufix<V>(q, bb[j], hw.items_bound, st);   // adjoint span entries
                if (r != cudaSuccess) return r;
                q.gb = gb;
                q.ga = ga;
                r = hi_reduce<V>(q, bb[j], st);
                timing_mark(kTimeUPass, 1, st);
                return r;
            });
            continue;
        }
        timing_mark(kTimeFused, 0, st);
        switch (p.lay[j].MB) {
#define X(V)                                                                                   \
    case V:                                                                                    \
        e = chunk_bwd_mb<V>(gy, x, y, b, a, saved, gx, gb, ga, gzi, tabs, counters + j, bb[j], \
                            p.lay[j].fp64_scan, read_y, three, num_sms, st);                   \
        break;
            DFILT_CHUNK_BUCKETS(X)
#undef X
            default: e = cudaErrorInvalidValue;
        }
        timing_mark(kTimeFused, 1, st);
    }
    timing_mark(1, 1, st);
    return e;
}

}  // namespace dfilt
