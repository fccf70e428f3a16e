// Host-side dispatch of the chunked algorithm: state-dimension bucket, scan precision,
// workspace sizes, and the setup + main kernel launches per bucket.
#include <cudaTypedefs.h>
#include <mutex>

#include "chunk.cuh"

namespace dfilt {

#define DFILT_EXTERN(V)                                                                          \
    extern template cudaError_t chunk_fwd_mb<V>(const float *, const float *, float *, float *, \
                                                const char *, const Batch &, bool, int, int,    \
                                                cudaStream_t);                                   \
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
    // filters, so the automatic choice is the FP64 scan there (and it is the only one
    // above the FP32 table bucket limit).
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

size_t chunk_fwd_ws_bytes(int64_t B, int Mmax, bool fp64_scan) {
    return kWsHeader + (size_t)B * chunk_layout(Mmax, fp64_scan ? 1 : 0).fwd_tab;
}

size_t chunk_bwd_ws_bytes(int64_t B, int Mmax, bool fp64_scan) {
    return kWsHeader + (size_t)B * chunk_layout(Mmax, fp64_scan ? 1 : 0).bwd_tab;
}

size_t chunk_saved_bytes(int64_t B, int64_t total, int Mmax, bool fp64_scan) {
    return chunk_saved_state_bytes(B, total, Mmax) +
           (size_t)B * chunk_layout(Mmax, fp64_scan ? 1 : 0).bwd_tab;
}

cudaError_t launch_chunk_fwd(const float *x, const float *b, const float *a, const float *zi,
                             float *y, float *saved, void *ws, const Batch &bt, int Mmax,
                             bool fp64_scan, int precision, int num_sms, cudaStream_t st) {
    const ChunkLayout l = chunk_layout(Mmax, fp64_scan ? 1 : 0);
    // with a saved buffer, the same launch also writes the backward's tables into it
    char *w = static_cast<char *>(ws);
    char *btabs = saved ? reinterpret_cast<char *>(saved) + chunk_saved_state_bytes(bt.B, bt.total, Mmax)
                        : nullptr;
    cudaError_t e = launch_chunk_setup(b, a, w + kWsHeader, btabs,
                                       reinterpret_cast<unsigned long long *>(w), bt, l.MB,
                                       l.fp64_scan, st);
    if (e != cudaSuccess) return e;
    const int three = precision == DFILT_PREC_TF32X3 ? 1 : 0;
    timing_mark(0, 0, st);
    switch (l.MB) {
#define X(V)                                                                        \
    case V: e = chunk_fwd_mb<V>(x, zi, y, saved, w, bt, l.fp64_scan, three, num_sms, st); \
        break;
        DFILT_CHUNK_BUCKETS(X)
#undef X
        default: e = cudaErrorInvalidValue;
    }
    timing_mark(0, 1, st);
    return e;
}

cudaError_t launch_chunk_bwd(const float *gy, const float *x, const float *y, const float *b,
                             const float *a, const float *saved, float *gx, float *gb, float *ga,
                             float *gzi, void *ws, const Batch &bt, int Mmax, bool fp64_scan,
                             int precision, int num_sms, cudaStream_t st) {
    const ChunkLayout l = chunk_layout(Mmax, fp64_scan ? 1 : 0);
    const bool read_y = saved == nullptr;   // y is recomputed whenever the chunk states exist
    if (read_y && (!y || l.MB > 32)) return cudaErrorNotSupported;
    char *wsc = static_cast<char *>(ws);
    auto *counter = reinterpret_cast<unsigned long long *>(wsc);
    const char *w;
    cudaError_t e;
    if (saved) {
        // the forward's setup left the backward tables behind the chunk states
        w = reinterpret_cast<const char *>(saved) + chunk_saved_state_bytes(bt.B, bt.total, Mmax);
        e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    } else {
        w = wsc + kWsHeader;
        e = launch_chunk_setup(b, a, nullptr, wsc + kWsHeader, counter, bt, l.MB, l.fp64_scan, st);
    }
    if (e != cudaSuccess) return e;
    const int three = precision == DFILT_PREC_TF32X3 ? 1 : 0;
    timing_mark(1, 0, st);
    switch (l.MB) {
#define X(V)                                                                                   \
    case V:                                                                                    \
        e = chunk_bwd_mb<V>(gy, x, y, b, a, saved, gx, gb, ga, gzi, w, counter, bt,            \
                            l.fp64_scan, read_y, three, num_sms, st);                          \
        break;
        DFILT_CHUNK_BUCKETS(X)
#undef X
        default: e = cudaErrorInvalidValue;
    }
    timing_mark(1, 1, st);
    return e;
}

}  // namespace dfilt
