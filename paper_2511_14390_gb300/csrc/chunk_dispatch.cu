// Host-side dispatch of the chunked algorithm: state-dimension bucket, scan precision,
// workspace sizes, and the setup + main kernel launches per bucket.
#include <cudaTypedefs.h>
#include <mutex>

#include "chunk.cuh"

namespace dfilt {

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
    // FP32 powers of the chunk transition stay stable for low orders; above order 4 the
    // transient growth of companion-matrix powers makes an FP32 scan diverge on some
    // filters, so the automatic choice there is the serial scan in double words
    // (FP64-class accuracy; the only one above the FP32 table bucket limit).
    l.fp64_scan = fp64_scan_opt < 0 ? (Mmax > 4) : (fp64_scan_opt != 0);
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

// Per-bucket plan: a fixed-shape batch is one bucket; a ragged batch runs every state
// bucket up to its largest order as its own launch pair (setup + main kernel) over the
// channels of that bucket, with records at a common stride.
ChunkPlan chunk_plan(int Mmax, int fp64_opt, bool ragged) {
    ChunkPlan p{};
    p.ragged = ragged;
    if (!ragged) {
        p.nb = 1;
        p.lay[0] = chunk_layout(Mmax, fp64_opt);
    } else {
        const int top = chunk_bucket(Mmax);
        p.nb = 0;
        for (int mb : {2, 4, 8, 16, 32, 64})
            if (mb <= top) p.lay[p.nb++] = chunk_layout(mb, fp64_opt);
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

size_t chunk_fwd_ws_bytes(int64_t B, int Mmax, int fp64_opt, bool ragged) {
    const ChunkPlan p = chunk_plan(Mmax, fp64_opt, ragged);
    return kWsHeader + (size_t)B * p.fstride + list_bytes(B, ragged);
}

size_t chunk_bwd_ws_bytes(int64_t B, int Mmax, int fp64_opt, bool ragged) {
    const ChunkPlan p = chunk_plan(Mmax, fp64_opt, ragged);
    return kWsHeader + (size_t)B * p.bstride + list_bytes(B, ragged);
}

size_t chunk_saved_bytes(int64_t B, int64_t total, int Mmax, int fp64_opt, bool ragged) {
    return chunk_saved_state_bytes(B, total, Mmax) + (size_t)B * chunk_plan(Mmax, fp64_opt, ragged).bstride;
}

namespace {

// Sort the channels of a ragged batch by state bucket (one block; order within a bucket
// is arbitrary, which no result depends on): list[starts[j] .. starts[j+1]) are the
// channels of bucket j (orders up to 2 << j; the last bucket takes the rest).
__global__ void __launch_bounds__(1024) bucket_channels_kernel(const int *__restrict__ Ms, int64_t B,
                                                               int Mstride, int nb,
                                                               int *__restrict__ list,
                                                               int *__restrict__ starts) {
    __shared__ int cnt[8], pos[8];
    if (threadIdx.x < 8) cnt[threadIdx.x] = 0;
    __syncthreads();
    auto bucket = [&](int64_t i) {
        int m = Ms[i];
        m = m < 1 ? 1 : (m > Mstride ? Mstride : m);
        int j = 0;
        while (j < nb - 1 && m > (2 << j)) ++j;
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

}  // namespace

cudaError_t launch_chunk_fwd(const float *x, const float *b, const float *a, const float *zi,
                             float *y, float *saved, void *ws, const Batch &bt, int Mmax,
                             int fp64_opt, int precision, int num_sms, cudaStream_t st) {
    const bool ragged = bt.offsets != nullptr && bt.Ms != nullptr;
    const ChunkPlan p = chunk_plan(Mmax, fp64_opt, ragged);
    char *w = static_cast<char *>(ws);
    auto *counters = reinterpret_cast<unsigned long long *>(w);   // one per bucket
    // with a saved buffer, the same setup launch also writes the backward's tables into it
    char *btabs = saved ? reinterpret_cast<char *>(saved) + chunk_saved_state_bytes(bt.B, bt.total, Mmax)
                        : nullptr;
    Batch bb[8];
    int *list = reinterpret_cast<int *>(w + kWsHeader + (size_t)bt.B * p.fstride);
    if (ragged) {
        bucket_channels_kernel<<<1, 1024, 0, st>>>(bt.Ms, bt.B, bt.Mstride, p.nb, list, list + bt.B);
        cudaError_t e = cudaGetLastError();
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
    for (int j = 0; j < p.nb && e == cudaSuccess; ++j) {
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
    }
    timing_mark(0, 1, st);
    return e;
}

cudaError_t launch_chunk_bwd(const float *gy, const float *x, const float *y, const float *b,
                             const float *a, const float *saved, float *gx, float *gb, float *ga,
                             float *gzi, void *ws, const Batch &bt, int Mmax, int fp64_opt,
                             int precision, int num_sms, cudaStream_t st) {
    const bool ragged = bt.offsets != nullptr && bt.Ms != nullptr;
    const ChunkPlan p = chunk_plan(Mmax, fp64_opt, ragged);
    const bool read_y = saved == nullptr;   // y is recomputed whenever the chunk states exist
    if (read_y && (!y || chunk_bucket(Mmax) > 32)) return cudaErrorNotSupported;
    char *wsc = static_cast<char *>(ws);
    auto *counters = reinterpret_cast<unsigned long long *>(wsc);   // one per bucket
    // the forward's setup left the backward tables behind the chunk states
    const char *tabs = saved ? reinterpret_cast<const char *>(saved) +
                                   chunk_saved_state_bytes(bt.B, bt.total, Mmax)
                             : wsc + kWsHeader;
    Batch bb[8];
    int *list = reinterpret_cast<int *>(wsc + kWsHeader + (size_t)bt.B * p.bstride);
    cudaError_t e = cudaSuccess;
    if (ragged) {
        bucket_channels_kernel<<<1, 1024, 0, st>>>(bt.Ms, bt.B, bt.Mstride, p.nb, list, list + bt.B);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (saved) e = cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * p.nb, st);
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
    for (int j = 0; j < p.nb && e == cudaSuccess; ++j) {
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
    }
    timing_mark(1, 1, st);
    return e;
}

}  // namespace dfilt
